"""Benchmark: priced instances per second of the AMFR-W2 sparse-grid solver.

Workload (one "step" = one batch): B seeded instances of the d=4 SABR-LMM
swaption problem (3 forward rates + V, standard combination level n=5, 121
component grids, 40 AMFR-W2 steps, FP64), each priced end to end (all
component grids, interpolation, combination).  Instances are sharded across
ranks with no collective on the data path (weak scaling).

  value  device-timed throughput with inputs resident in HBM (CUDA events
         on the library's stream around each batch; L2 flushed between
         batches by a 256 MiB write outside the timed events)
  e2e    the same metric through the C-ABI call amfrw_solve_batch with host
         buffers (validation, grid enumeration, upload, solve, download)
  roofline  the dominant solver kernel: algorithmic FP64 FLOPs of its launch
         (counted per node from Sketch 1 and the Thomas sweeps) / its CUDA
         event duration, against the FP64 peak derived from 152 SMs x
         2 DFMA/clk x 2070 MHz
  cpu_baseline  the CPU oracle on the host cores (bounded sample)

--impl reference runs the oracle arm instead (the reference of this build is
the plain FP64 CPU implementation of the paper's method).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2408_00559_gb300 import workloads as W  # noqa: E402

METRIC = "priced instances/sec at 1e-5 rel. error (batched/mixed vs plain; surrogate)"
UNIT = "instances/s"
WORKLOAD = ("c2: d=4 (3 forward rates + V) SABR-LMM swaption, standard combination level 5 "
            "(121 component grids, 15149 nodes), 40 AMFR-W2 steps, T=2, FP64")
FP64_PEAK = 152 * 2 * 2 * 2070e6  # SMs x DFMA/clk x FLOP/FMA x max SM clock
FP32_PEAK = 152 * 128 * 2 * 2070e6  # SMs x FFMA/clk x FLOP/FMA x max SM clock
WORKLOADS = {
    "c2": dict(desc=WORKLOAD, d=4, n=5, psi=0, dtype="f64", batch=4096),
    "c3": dict(desc=("c3: d=6 (5 forward rates + V) swaption, modified combination psi=1 level 6 "
                     "(923 grids, 13.5 M nodes), 40 steps, mixed FP32/FP64"),
               d=6, n=6, psi=1, dtype="f32+f64", batch=4),
    "c4": dict(desc=("c4: d in {4,6,8}, level in {4,5,6}, standard combination, 40 steps, "
                     "mixed FP32/FP64"), d=None, n=None, psi=0, dtype="f32+f64", batch=256),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=None, help="instances per step per GPU")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4"],
                    help="c2 (default, the metric's configuration); c3/c4 for profiling runs")
    return ap.parse_args()


# ---------------------------------------------------------------- FLOP count
def node_flops(levels, steps):
    """Algorithmic FP64 FLOPs of one component grid over `steps` AMFR-W2
    steps (FMA = 2).  Per F evaluation at an Inner node (Sketch 1 with the
    coefficients from per-axis tables): 3 per second difference, 1 per
    gradient of a drift axis not on its upper face, for each pair (i,k) with
    both indices below their upper faces 3 for the cross difference plus 3
    (rate pair: table product and FMA) or 2 (pair with V), per drift axis
    2i+3 when not on its upper face, 2 per rate axis for the outer
    coefficient FMA and 2(N-1)+1 for the diagonal coefficients; 4 F
    evaluations per step plus 4 (stage-argument) and 5 (refinement) per
    node for the fused stage algebra, 5 per row of each of the 4N Thomas
    sweeps, and 6 for the two fused updates."""
    N = len(levels)
    M = [1 << int(l) for l in levels]
    axes = [np.arange(1, m + 1) for m in M]
    grids = np.meshgrid(*axes, indexing="ij")
    top = [grids[i] == M[i] for i in range(N)]
    nt = [~t for t in top]
    f = np.full(grids[0].shape, 3 * N + 1 + 2 * (N - 1) + 2 * (N - 1), dtype=np.float64)
    for i in range(1, N - 1):  # drift axes
        f += nt[i] * (1 + 2 * i + 3)
    for i in range(N - 1):
        for k in range(i + 1, N):
            both = nt[i] & nt[k]
            f += both * (3 + (3 if k < N - 1 else 2))
    per_step = 4 * f.sum() + f.size * (2 * 4 + 2 * 5 + 20 * N + 6)
    return float(per_step) * steps


def c2_flops_per_instance():
    from paper_2408_00559_gb300._lib import Problem  # noqa: F401  (shapes only below)
    lv = enumerate_levels(4, 5, 0)
    return sum(node_flops(l, 40) for l in lv)


def enumerate_levels(d, n, psi):
    out = []

    def rec(prefix, m):
        if len(prefix) == d - 1:
            out.append(prefix + [m])
            return
        for v in range(m + 1):
            rec(prefix + [v], m - v)

    for q in range(d):
        if n - q >= 0:
            rec([], n - q)
    return [[psi + x for x in l] for l in out]


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle
def _oracle_price(inst):
    import oracle as O
    return O.price(inst, inst["level"], inst["psi"], inst.get("full", False))


def cpu_oracle_rate(seconds: float, start: int):
    """The oracle as it stands, one instance per worker process, all host
    cores, for about `seconds` of wall time.  Returns (instances/s, cores,
    instances done)."""
    import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    done = 0
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        idx = start
        while True:
            chunk = W.batch("c2", cores, start=idx)
            idx += cores
            pool.map(_oracle_price, chunk)
            done += len(chunk)
            if time.perf_counter() - t0 >= seconds:
                break
    dt = time.perf_counter() - t0
    return done / dt, cores, done


# ------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    # each step prices one chunk of instances on all host cores
    import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        for w in range(args.warmup):
            pool.map(_oracle_price, W.batch("c2", cores, start=10_000_000 + w * cores))
        t0 = time.perf_counter()
        for k in range(args.steps):
            pool.map(_oracle_price, W.batch("c2", cores, start=k * cores))
        dt = time.perf_counter() - t0
    value = args.steps * cores / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch": cores, "impl": "CPU oracle (plain serial FP64 C, "
                   "one instance per process)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps x {cores} c2 instances"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2408_00559_gb300 import _lib as L
    from paper_2408_00559_gb300 import build as BLD

    # CPU baseline first (spawned pool, before any GPU call)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, done = cpu_oracle_rate(args.cpu_seconds, start=20_000_000)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{done} c2 instances, one per process on {cores} host cores, "
                         f"~{args.cpu_seconds:.0f} s"}

    BLD.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    wl = WORKLOADS[args.workload]
    B = args.batch or wl["batch"]
    insts = W.batch(args.workload, B, start=rank * B)
    with torch.cuda.stream(stream):
        batch = L.Batch(insts, stream=stream)
        batch.enable_timing(True)
        prices = torch.empty(B, dtype=torch.float64, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        n_launch = batch.launches()
        for _ in range(args.warmup):
            batch.run(prices.data_ptr())
        stream.synchronize()
        # accuracy of the priced instances against the oracle (sampled)
        check = {"oracle_checked": 0, "note": "covered by the GPU parity tests"}
        if rank == 0 and args.workload == "c2":
            import oracle as O
            got = prices.cpu().numpy()
            rel = []
            for i in (0, B // 2, B - 1):
                po = O.price(insts[i], 5)
                rel.append(abs(got[i] - po) / abs(po))
            check = {"oracle_checked": 3, "max_rel_err": max(rel), "tolerance": 1e-12}
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        ktimes = []
        with ClockSampler(local_rank) as clk:
            for k in range(args.steps):
                flush.fill_(k & 0xFF)
                evs[k][0].record(stream)
                batch.run(prices.data_ptr())
                evs[k][1].record(stream)
                ktimes.append(batch.kernel_times())
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        step_ms = [s.elapsed_time(e) for s, e in evs]
    total_s = sum(step_ms) / 1e3
    if world > 1:
        t = torch.tensor([total_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_s = float(t.item())
    value = world * B * args.steps / total_s

    # dominant kernel: the solver kernel, launched once per (N, grid-size)
    # class; all its launches of one batch together form its work for the batch
    launches_per_batch = len(ktimes[0])
    kernel_ms = [sum(ms for (N, ms, ns) in kt) for kt in ktimes]
    avg_ms = sum(kernel_ms) / len(kernel_ms)
    flops_batch = 0.0
    shapes = {}
    for inst in insts:
        key = (inst["N"], inst["level"], inst["psi"])
        if key not in shapes:
            shapes[key] = sum(node_flops(l, inst["n_steps"]) for l in enumerate_levels(*key))
        flops_batch += shapes[key]
    achieved = flops_batch / (avg_ms / 1e3)
    fp64 = wl["dtype"] == "f64"
    peak = FP64_PEAK if fp64 else FP32_PEAK

    # end to end through the C ABI with host buffers
    h2d, d2h = batch.io_bytes()
    m = L._Marshal(insts)
    host_prices = np.zeros(B)
    lib = L.lib()
    sptr = int(stream.cuda_stream)
    for _ in range(max(1, args.warmup // 2)):
        L._check(lib.amfrw_solve_batch(m.arr, B, L._dp(host_prices), sptr), "amfrw_solve_batch")
    e2e_steps = max(2, args.steps // 2)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        L._check(lib.amfrw_solve_batch(m.arr, B, L._dp(host_prices), sptr), "amfrw_solve_batch")
    e2e_s = time.perf_counter() - t0
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert np.array_equal(host_prices, prices.cpu().numpy()), "e2e prices differ from the device run"
    batch.close()

    if rank != 0:
        return
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl["dtype"], "data": "synthetic",
        "config": {"workload": wl["desc"], "batch_per_gpu": B,
                   "parallelism": f"dp{world} (instances sharded, no collective)",
                   "l2": "flushed between timed batches (256 MiB write outside the events)"},
        "roofline": {"bound": "alu", "pipe": "fp64" if fp64 else "fp32",
                     "kernel": "solve_kernel (all per-class launches of a batch)",
                     "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel_ms_per_batch": avg_ms, "solver_launches_per_batch": launches_per_batch,
                     "flops_per_batch": flops_batch,
                     "peak_source": ("derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2070 MHz" if fp64 else
                                     "derived: 152 SMs x 128 FFMA/clk x 2 FLOP x 2070 MHz")},
        "cpu_baseline": cpu,
        "e2e": {"value": world * B * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": n_launch * args.steps,
        "clocks": clocks,
        "parity": check,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
