"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

FP64 path: every Inner node of every component grid, the interpolated value
of every grid and the combined price agree with the oracle to 1e-12
relative (node values relative to the grid's largest value; prices relative
to the price).  Mixed path (FP32 stencil and line solves, FP64 accumulation,
interpolation and combination): prices to 1e-5 relative, grid values to
1e-6 relative to the grid's largest value.

Cases cover N = 2..8, standard / modified / full grids, caplet and swaption,
both work-group kinds (one warp for grids of <= 256 Inner nodes, a whole
CTA above), degenerate axes (M_i = 1), levels below d-1 (few grids), the
spot on the Neumann face, a single step, beta = 0 and 1, sigma = 0.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX_PRICE = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


def inner(Y_full, levels):
    shape = tuple((1 << int(l)) + 1 for l in reversed(levels))
    A = Y_full.reshape(shape)
    return A[(slice(1, None),) * len(levels)].ravel()


def oracle_grids(inst):
    lv, cf = O.enumerate_grids(inst["N"], inst["level"], inst.get("psi", 0), inst.get("full", False))
    return {tuple(int(x) for x in l): (k, c) for k, (l, c) in enumerate(zip(lv, cf))}


def check_problem(inst, tol_node, tol_price, sample=None):
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    p_gpu = prob.combine()
    lv, cf = prob.grid_info()
    u_gpu = prob.grid_values()
    og = oracle_grids(inst)
    assert len(og) == len(lv)
    idx = range(len(lv)) if sample is None else sample
    for g in idx:
        key = tuple(int(x) for x in lv[g])
        assert key in og
        assert cf[g] == og[key][1]
        u_o, Yf = O.solve_grid(inst, lv[g], want_Y=True)
        Yo = inner(Yf, lv[g])
        Yg = prob.read_grid(g, lv[g])
        scale = max(np.max(np.abs(Yo)), 1e-300)
        err = np.max(np.abs(Yg - Yo)) / scale
        assert err <= tol_node, (key, err)
        assert abs(u_gpu[g] - u_o) <= tol_node * scale, (key, u_gpu[g], u_o)
    if sample is None:
        p_o = O.price(inst, inst["level"], inst.get("psi", 0), inst.get("full", False))
        assert abs(p_gpu - p_o) <= tol_price * abs(p_o), (p_gpu, p_o)
    prob.close()
    return p_gpu


def test_c1_full_grid_65x65_fp64():
    check_problem(W.c1_instance(), TOL64, TOL64)


def test_c2_d4_standard_n5_fp64_all_grids():
    check_problem(W.c2_instance(0), TOL64, TOL64)


CASES = [
    # (N, level, psi, full, payoff, steps)
    (2, 5, 0, False, "caplet", 6),
    (2, 4, 2, False, "swaption", 3),
    (3, 4, 0, False, "swaption", 5),
    (3, 3, 1, False, "caplet", 4),
    (3, 4, 0, True, "swaption", 2),       # 16^3 = 4096 Inner nodes: CTA group
    (4, 2, 1, False, "swaption", 3),      # grids of 2^6..2^8 nodes
    (5, 3, 0, False, "swaption", 3),
    (6, 2, 1, False, "swaption", 2),      # modified, CTA groups of 2^8..2^8
    (7, 3, 0, False, "swaption", 2),
    (8, 4, 0, False, "swaption", 2),
    (8, 1, 0, False, "swaption", 3),      # level below d-1: only q <= 1 grids
    (4, 0, 0, False, "swaption", 2),      # all axes degenerate (M_i = 1)
    (4, 7, 0, False, "swaption", 2),      # CTA groups (128 nodes) with single-row axes: folded solves
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0]}_n{c[1]}_psi{c[2]}_{'full' if c[3] else 'sg'}_{c[4]}" for c in CASES])
def test_fp64_cases(case):
    N, n, psi, full, payoff, steps = case
    inst = W.small_instance(N, n, psi=psi, steps=steps, seed=N * 100 + n, full=full, payoff=payoff)
    check_problem(inst, TOL64, TOL64)


@pytest.mark.parametrize("variant", ["beta0", "beta1", "sigma0", "spot_inside", "one_step", "discount"])
def test_fp64_parameter_edges(variant):
    inst = W.small_instance(4, 3, steps=4, seed=7)
    if variant == "beta0":
        inst["beta"] = 0.0
    elif variant == "beta1":
        inst["beta"] = 1.0
    elif variant == "sigma0":
        inst["sigma"] = 0.0
    elif variant == "spot_inside":
        inst["V0"] = 0.37
        inst["F0"] = np.array([0.011, 0.047, 0.083])
    elif variant == "one_step":
        inst["n_steps"] = 1
    elif variant == "discount":
        inst["discount"] = 0.97
    check_problem(inst, TOL64, TOL64)


def test_paper_caplet_table_on_gpu():
    # Table fg_sigma0, level 6, 4 time steps: 6.084214 bps (nu = theta for N = 2)
    th = (3 + math.sqrt(3)) / 6
    inst = dict(N=2, payoff="caplet", n_steps=4, alpha=[0.2366], phi=[0.0], tau=[0.5], F0=[0.0118],
                Fmax=[0.04], Vmax=3.5, rho=np.ones((1, 1)), sigma=0.0, beta=1.0, V0=1.0, K=0.011,
                T=0.5, theta=th, nu=th, discount=1.0, level=6, psi=0, full=True, precision="fp64")
    u = B.solve_batch([inst])[0]
    bps = 1e4 * 0.5 * u / ((1 + 0.5 * 0.0112) * (1 + 0.5 * 0.0118))
    assert abs(bps - 6.084214) < 5.5e-7


def test_step_is_resumable():
    inst = W.small_instance(3, 4, steps=8, seed=11)
    a = B.Problem(inst)
    a.step(8)
    b = B.Problem(inst)
    b.step(3)
    b.step(5)
    assert abs(a.combine() - b.combine()) <= 1e-14 * max(1.0, abs(a.combine()))


@pytest.mark.parametrize("case", [(4, 3), (4, 7)], ids=["warp_groups", "cta_groups"])
def test_mixed_step_is_resumable(case):
    """Mixed precision across amfrw_step calls: the state keeps Y in FP64 and
    the next call rebuilds Z and its float pair from it (CTA groups keep Z in
    their block's global slice), so the split run follows the uninterrupted
    one to far below the mode's FP32 rounding."""
    N, n = case
    inst = W.small_instance(N, n, steps=8, seed=13, precision="mixed")
    a = B.Problem(inst)
    a.step(8)
    b = B.Problem(inst)
    b.step(3)
    b.step(5)
    pa, pb = a.combine(), b.combine()
    assert abs(pa - pb) <= 1e-9 * abs(pa), (pa, pb)
    po = O.price(inst, n, 0)
    assert abs(pb - po) <= TOLMIX_PRICE * abs(po), (pb, po)


def test_batch_equals_single_problems_and_is_deterministic():
    insts = W.batch("c2", 6)
    p1 = B.solve_batch(insts)
    p2 = B.solve_batch(insts)
    assert np.array_equal(p1, p2)
    for i, inst in enumerate(insts[:3]):
        pr = B.Problem(inst)
        pr.step(inst["n_steps"])
        assert abs(pr.combine() - p1[i]) <= TOL64 * abs(p1[i])


def test_batch_run_into_device_tensor():
    import torch
    insts = W.batch("c2", 8, start=100)
    b = B.Batch(insts)
    out = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    b.run(out.data_ptr())
    torch.cuda.synchronize()
    ref = B.solve_batch(insts)
    assert np.array_equal(out.cpu().numpy(), ref)
    assert b.launches() >= 2


def test_c2_batch_sampled_against_oracle():
    insts = W.batch("c2", 64, start=1000)
    p = B.solve_batch(insts)
    for i in (0, 17, 63):
        po = O.price(insts[i], 5)
        assert abs(p[i] - po) <= TOL64 * abs(po), (i, p[i], po)


# ------------------------------------------------------------------ mixed
@pytest.mark.parametrize("case", [(4, 3, 0), (6, 2, 1), (8, 3, 0), (3, 4, 1), (4, 7, 0)],
                         ids=["N4_n3", "N6_n2_psi1", "N8_n3", "N3_n4_psi1", "N4_n7_cta"])
def test_mixed_precision_price(case):
    N, n, psi = case
    inst = W.small_instance(N, n, psi=psi, steps=10, seed=500 + N, precision="mixed")
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    p = prob.combine()
    po = O.price(inst, n, psi)
    assert abs(p - po) <= TOLMIX_PRICE * abs(po), (p, po, abs(p - po) / abs(po))
    lv, _ = prob.grid_info()
    for g in (0, len(lv) // 2, len(lv) - 1):
        Yo = inner(O.solve_grid(inst, lv[g], want_Y=True)[1], lv[g])
        Yg = prob.read_grid(g, lv[g])
        assert np.max(np.abs(Yg - Yo)) <= 1e-6 * np.max(np.abs(Yo))


def test_c3_full_size_sampled_grids():
    """d=6 modified psi=1 n=6 (923 grids, up to 4096 Inner nodes), mixed
    precision: sampled component grids against the oracle one by one, and
    the price against the oracle's price of the whole problem (all 923 grids,
    solved by the oracle in a spawned process pool) at 1e-5."""
    inst = W.c3_instance(0)
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    lv, cf = prob.grid_info()
    u = prob.grid_values()
    sizes = np.array([np.prod([(1 << int(x)) for x in l]) for l in lv])
    pick = [int(np.argmax(sizes)), int(np.argmin(sizes)), len(lv) // 3]
    for g in pick:
        u_o, Yf = O.solve_grid(inst, lv[g], want_Y=True)
        Yo = inner(Yf, lv[g])
        Yg = prob.read_grid(g, lv[g])
        assert np.max(np.abs(Yg - Yo)) <= 1e-6 * np.max(np.abs(Yo)), lv[g]
        assert abs(u[g] - u_o) <= 1e-6 * np.max(np.abs(Yo))
    p = prob.combine()
    prob.close()
    po = O.price_parallel(inst, inst["level"], inst["psi"])
    assert abs(p - po) <= TOLMIX_PRICE * abs(po), (p, po, abs(p - po) / abs(po))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_c4_full_size_d8_sampled_grids(precision):
    """The largest shape of the batched workload, d=8 standard level 6 (3003
    grids of 256..8320 nodes, 40 steps), taken from the 256-instance batch:
    sampled component grids against the oracle one by one (the largest, the
    smallest, and the one with the most refined axes, which has the most
    active cross and drift terms), node by node."""
    inst = dict(W.batch("c4", 2)[1], precision=precision)
    assert inst["N"] == 8 and inst["level"] == 6
    tol = TOL64 if precision == "fp64" else 1e-6
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    lv, cf = prob.grid_info()
    u = prob.grid_values()
    assert len(lv) == 3003
    sizes = np.array([np.prod([(1 << int(x)) + 1 for x in l]) for l in lv])  # with Outer nodes
    spread = np.array([np.count_nonzero(l) for l in lv])
    pick = [int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argmax(spread))]
    for g in pick:
        u_o, Yf = O.solve_grid(inst, lv[g], want_Y=True)
        Yo = inner(Yf, lv[g])
        Yg = prob.read_grid(g, lv[g])
        scale = np.max(np.abs(Yo))
        assert np.max(np.abs(Yg - Yo)) <= tol * scale, (lv[g], np.max(np.abs(Yg - Yo)) / scale)
        assert abs(u[g] - u_o) <= tol * scale, (lv[g], u[g], u_o)
    assert np.isfinite(prob.combine())
    prob.close()
