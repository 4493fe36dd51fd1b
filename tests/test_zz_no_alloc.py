"""amfrw_solve_noalloc, the entry point for callers that cannot allocate
device memory (their memory belongs to another allocator, or they cannot
afford cudaMalloc/cudaFree and the device-wide synchronisation of a free).

It must price exactly like amfrw_solve_batch, the allocating entry point, and
keep doing so on a second call in a row, because every call reuses the same
fixed device array and inherits the previous call's contents.  Four problem
sets are used: d=4 level-5 swaptions (grids solved one per warp), the 65x65
full grid in FP64 (solved by a whole block, whose line-solve factors live in
the fixed array), a small d=6 modified problem in mixed precision, and the
largest problem the header promises to fit: one d=6 (5 rates + V) modified
psi=1 level-6 instance in mixed precision (923 grids of up to 4096 Inner
nodes, solved by whole blocks with their factors in the array).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


@pytest.mark.parametrize("which", ["c2_batch", "c1_full_grid", "mixed_d6", "c3_d6_level6"])
def test_noalloc_matches_allocating_entry_point_twice(which):
    import torch
    if which == "c2_batch":
        insts = W.batch("c2", 48, start=321)
    elif which == "c1_full_grid":
        insts = [W.c1_instance()]
    elif which == "mixed_d6":
        insts = [W.small_instance(6, 3, psi=1, steps=5, seed=9, precision="mixed")]
    else:
        insts = W.batch("c3", 1, start=17)
    ref = B.solve_batch(insts)
    out = torch.full((len(insts),), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(float("nan"))
        B.solve_noalloc(insts, out.data_ptr())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert np.all(np.abs(got - ref) <= TOL64 * np.abs(ref)), (call, got - ref)


def test_noalloc_rejects_problems_beyond_its_array():
    import torch
    insts = W.batch("c2", 4000)  # needs more than AMFRW_NOALLOC_SCRATCH_BYTES
    out = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    with pytest.raises(B.AmfrwError) as e:
        B.solve_noalloc(insts, out.data_ptr())
    assert e.value.status == 7 and "limited to" in str(e.value)


def test_noalloc_refuses_to_be_captured_into_a_graph():
    # its records come from host buffers freed on return, so a graph replay
    # would read freed memory: the call must refuse while its stream captures
    import torch
    insts = W.batch("c2", 2, start=5)
    out = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            with pytest.raises(B.AmfrwError) as e:
                B.solve_noalloc(insts, out.data_ptr(), stream=s)
        finally:
            g.capture_end()
    assert e.value.status == 1 and "captured" in str(e.value)
