"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): ranks
price disjoint blocks of seeded instances that together are the one-rank
batch, the job time is the slowest rank's, and the job rate counts every
rank's instances.  The instances are priced by the CPU oracle here, so the
test needs no GPU."""
import os
import socket

import numpy as np
import torch.multiprocessing as tmp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, per_rank, out):
    import torch.distributed as dist

    import bench
    import oracle as O
    from paper_2408_00559_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start = bench.shard_start(rank, per_rank)
    insts = W.batch("c2", per_rank, start=start)
    for x in insts:
        x["n_steps"] = 2
    prices = [O.price(x, x["level"], 0) for x in insts]
    seconds = 1.0 + rank  # rank 1 is the slower one
    t = bench.max_over_ranks(seconds, world, "cpu")
    gathered = [None] * world
    dist.all_gather_object(gathered, (start, prices))
    if rank == 0:
        out.put((t, gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_time_like_one():
    world, per_rank = 2, 2
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, per_rank, q)) for r in range(world)]
    for p in procs:
        p.start()
    t, gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 2.0
    starts = [g[0] for g in gathered]
    assert starts == [0, per_rank]
    # the two shards are the one-rank batch of 2 * per_rank instances
    import bench
    import oracle as O
    from paper_2408_00559_gb300 import workloads as W
    whole = W.batch("c2", world * per_rank, start=0)
    for x in whole:
        x["n_steps"] = 2
    ref = [O.price(x, x["level"], 0) for x in whole]
    got = [p for g in gathered for p in g[1]]
    assert np.array_equal(np.array(got), np.array(ref))
    assert bench.job_rate(world, per_rank, 10, t) == world * per_rank * 10 / 2.0
