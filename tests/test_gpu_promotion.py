"""GPU tests of the FP64 re-solve of ill-conditioned mixed-precision instances.

A mixed-precision price is accurate relative to the combination's scale
sum_l |c_l u_l|, not to the price itself; where the combination sum cancels
(kappa = sum_l |c_l u_l| / |price| large) the batch re-solves the instance in
FP64 inside its CUDA graph.  The tests check:
- kappa as the library reports it against kappa recomputed from the FP64
  grid values of the same instance (the Problem entry point);
- a bound below every kappa re-solves every instance: the prices are then the
  FP64 prices;
- a bound above every kappa re-solves nothing: the prices are the plain mixed
  ones, bitwise;
- with the default bound every price of the d=4 level-5 batch (4096
  instances, some of whose combination sums cancel to 1e-6 against a scale of
  4) is within 1e-5 of its FP64 price.
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


def run(insts, kappa_max=None):
    import torch
    b = B.Batch(insts)
    if kappa_max is not None:
        b.set_kappa_max(kappa_max)
    out = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    b.run(out.data_ptr())
    torch.cuda.synchronize()
    n, kappa = b.promoted()
    p = out.cpu().numpy().copy()
    b.close()
    return p, n, kappa


def test_kappa_is_the_condition_of_the_combination_sum():
    insts = [dict(x, precision="mixed") for x in W.batch("c2", 6, start=40)]
    _, _, kappa = run(insts)
    for i in (0, 3, 5):
        x = dict(insts[i], precision="fp64")
        pr = B.Problem(x)
        pr.step(x["n_steps"])
        _, cf = pr.grid_info()
        cu = np.asarray(cf) * pr.grid_values()
        pr.close()
        ref = np.sum(np.abs(cu)) / abs(np.sum(cu))
        # kappa comes from the mixed grid values: it agrees to their accuracy
        assert abs(kappa[i] - ref) <= 1e-4 * ref, (i, kappa[i], ref)


def test_bound_below_every_kappa_gives_the_fp64_prices():
    insts = W.batch("c4", 12, start=300)
    for x in insts:
        x["n_steps"] = 8
    p_all, n_all, kappa = run(insts, kappa_max=0.5)  # kappa >= 1 always
    assert n_all == len(insts)
    p64, _, _ = run([dict(x, precision="fp64") for x in insts])
    assert np.all(np.abs(p_all - p64) <= 1e-12 * np.abs(p64)), np.max(np.abs(p_all - p64) / np.abs(p64))


def test_bound_above_every_kappa_changes_nothing():
    insts = W.batch("c4", 12, start=300)
    for x in insts:
        x["n_steps"] = 8
    p_off, n_off, _ = run(insts, kappa_max=0.0)
    p_hi, n_hi, kappa = run(insts, kappa_max=1e300)
    assert n_off == 0 and n_hi == 0
    assert np.array_equal(p_off, p_hi)
    # and the default bound re-solves exactly the instances above it
    p_def, n_def, kappa_def = run(insts)
    assert n_def == int(np.sum(kappa_def > 1e5))


def test_default_bound_meets_1e5_on_every_instance_of_the_d4_batch():
    insts = W.batch("c2", 4096, start=0)
    p64, _, _ = run(insts)
    pm, n, kappa = run([dict(x, precision="mixed") for x in insts])
    rel = np.abs(pm - p64) / np.abs(p64)
    assert rel.max() <= 1e-5, (rel.max(), int(rel.argmax()), kappa[int(rel.argmax())], n)
    assert n == int(np.sum(kappa > 1e5))
