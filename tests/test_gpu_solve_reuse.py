"""amfrw_solve_batch keeps its last plan per thread (grid list, device
buffers, captured graph) and reuses it for a call whose instances have the
same shapes: such a call only uploads the new parameter records.  The reused
plan must price exactly like a fresh one, for new parameters, in both
precisions (the mixed batch carries its FP64 re-solve plan too), and any
change of shape, stream or an explicit release must plan afresh.
"""
import numpy as np
import pytest

from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


def fresh(insts):
    """Prices from a plan built for this call alone."""
    B.solve_batch_release()
    p = B.solve_batch(insts)
    B.solve_batch_release()
    return p


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_reused_plan_prices_new_parameters_like_a_fresh_plan(precision):
    a = W.batch("c4", 24, start=500, precision=precision)
    # the same shapes with other parameters: strike, volatility of volatility
    # and spot volatility moved
    b = [dict(x, K=x["K"] * 1.1, sigma=x["sigma"] * 0.8, V0=x["V0"] * 0.9) for x in a]
    pa, pb = fresh(a), fresh(b)
    assert not np.array_equal(pa, pb)
    B.solve_batch_release()
    q1 = B.solve_batch(a)
    h2d_first, d2h = B.solve_batch_io()
    q2 = B.solve_batch(b)          # reuses a's plan
    h2d_reuse, d2h2 = B.solve_batch_io()
    q3 = B.solve_batch(a)          # and back
    B.solve_batch_release()
    assert np.array_equal(q1, pa)
    assert np.array_equal(q2, pb)
    assert np.array_equal(q3, pa)
    # a reused plan uploads the instance records only (both plans when mixed)
    assert 0 < h2d_reuse < h2d_first
    assert d2h == d2h2 == 8 * len(a) + 4


def test_shape_change_stream_change_and_release_plan_afresh():
    import torch
    a = W.batch("c4", 12, start=40)
    c = W.batch("c4", 12, start=41)   # shifted: other shapes in the same positions
    assert [(x["N"], x["level"]) for x in a] != [(y["N"], y["level"]) for y in c]
    pa, pc = fresh(a), fresh(c)
    B.solve_batch_release()
    B.solve_batch(a)
    h_first, _ = B.solve_batch_io()
    assert np.array_equal(B.solve_batch(c), pc)
    assert B.solve_batch_io()[0] == fresh_io(c)
    s = torch.cuda.Stream()
    assert np.array_equal(B.solve_batch(c, stream=s), pc)   # another stream: a fresh plan
    assert B.solve_batch_io()[0] == fresh_io(c)
    B.solve_batch(a)
    B.solve_batch_release()
    assert np.array_equal(B.solve_batch(a), pa)             # released: a fresh plan
    assert B.solve_batch_io()[0] == h_first
    B.solve_batch_release()


def fresh_io(insts):
    b = B.Batch(insts)
    h, _ = b.io_bytes()
    b.close()
    return h


def test_reused_plan_still_validates_parameters():
    a = W.batch("c4", 6, start=7)
    B.solve_batch_release()
    B.solve_batch(a)
    bad = [dict(x) for x in a]
    bad[3]["V0"] = -1.0
    with pytest.raises(RuntimeError, match="instance 3"):
        B.solve_batch(bad)
    # the kept plan is still usable
    assert np.array_equal(B.solve_batch(a), fresh(a))
