"""GPU parity of the global-memory work groups: component grids whose state
does not fit in shared memory, or whose lines are longer than 256 rows, are
solved by one CTA with the grid in its slice of global scratch and the line
solves streamed from memory.

- Forced onto that path (AMFRW_FLAG_GLOBAL_GRIDS), the parity cases of the
  shared-memory path agree with the oracle node by node to 1e-12 (FP64) and
  in price to 1e-5 (mixed).
- Large grids take it by themselves: full grids of 129^2 and 257^2 nodes,
  a d=3 full grid of 2^21 Inner nodes, a d=3 combination with 512-row lines,
  against the oracle node by node.
- Every caplet value the paper prints (Tables fg_sigma0, fg_2d, d2_1,
  d1_sg_sigma, d1:Level; the oracle reproduces all of them) is reproduced on
  the GPU, including the rows that need this path.
- Steps resume across calls; a batch mixing small and large grids equals
  the single problems.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W
from test_gpu_parity import TOL64, TOLMIX_PRICE, check_problem, inner

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_tables.json")))
MKT = GOLD["market"]
THETA = (3 + math.sqrt(3)) / 6


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


FORCED = [
    # (N, level, psi, full, payoff, steps)
    (2, 5, 0, False, "caplet", 6),
    (3, 4, 0, True, "swaption", 2),
    (4, 3, 0, False, "swaption", 3),
    (5, 3, 0, False, "swaption", 2),
    (6, 2, 1, False, "swaption", 2),
    (8, 2, 0, False, "swaption", 2),
    (4, 0, 0, False, "swaption", 2),  # every axis degenerate (M_i = 1)
]


@pytest.mark.parametrize("case", FORCED, ids=[f"N{c[0]}_n{c[1]}_psi{c[2]}" + ("_full" if c[3] else "") for c in FORCED])
def test_forced_global_path_fp64(case):
    N, n, psi, full, payoff, steps = case
    inst = W.small_instance(N, n, psi=psi, steps=steps, seed=N * 100 + n, full=full, payoff=payoff)
    inst["global_grids"] = True
    check_problem(inst, TOL64, TOL64)


def test_forced_global_path_c1():
    check_problem(dict(W.c1_instance(), global_grids=True), TOL64, TOL64)


@pytest.mark.parametrize("case", [(4, 3, 0), (6, 2, 1), (3, 4, 1)], ids=["N4_n3", "N6_n2_psi1", "N3_n4_psi1"])
def test_forced_global_path_mixed(case):
    N, n, psi = case
    inst = W.small_instance(N, n, psi=psi, steps=10, seed=500 + N, precision="mixed")
    inst["global_grids"] = True
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    p = prob.combine()
    po = O.price(inst, n, psi)
    assert abs(p - po) <= TOLMIX_PRICE * abs(po), (p, po)
    prob.close()


@pytest.mark.parametrize("level,steps", [(7, 6), (8, 3)])
def test_large_full_grids(level, steps):
    inst = dict(W.c1_instance(), level=level, n_steps=steps)
    check_problem(inst, TOL64, TOL64)


def test_grid_of_two_million_inner_nodes():
    # d=3 full grid of level 7: 128^3 = 2^21 Inner nodes (above 2^20)
    inst = W.small_instance(3, 7, steps=2, seed=21, full=True, payoff="swaption")
    check_problem(inst, TOL64, TOL64)


def test_long_lines_d3_standard_level9():
    # axes of up to 2^9 = 512 rows
    inst = W.small_instance(3, 9, steps=4, seed=9, payoff="swaption")
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    p = prob.combine()
    lv, _ = prob.grid_info()
    longest = [g for g in range(len(lv)) if max(lv[g]) == 9]
    assert longest
    for g in longest[:2] + [len(lv) // 2]:
        Yo = inner(O.solve_grid(inst, lv[g], want_Y=True)[1], lv[g])
        Yg = prob.read_grid(g, lv[g])
        assert np.max(np.abs(Yg - Yo)) <= TOL64 * np.max(np.abs(Yo)), lv[g]
    po = O.price(inst, 9, 0)
    assert abs(p - po) <= TOL64 * abs(po), (p, po)
    prob.close()


def caplet(case):
    return dict(N=2, payoff="caplet", n_steps=case["steps"], alpha=[MKT["alpha"][1]], phi=[case["phi"]],
                tau=[MKT["tau"]], F0=[MKT["F0"][1]], Fmax=[MKT["Fmax"]], Vmax=MKT["Vmax"],
                rho=np.ones((1, 1)), sigma=case["sigma"], beta=MKT["beta"], V0=MKT["V0"], K=MKT["K"],
                T=MKT["T"][1], theta=THETA, nu=THETA, discount=1.0, level=case["level"],
                psi=case.get("psi", 0), full=case["grid"] == "full", precision="fp64")


def test_every_printed_caplet_value_on_gpu():
    P2 = 1.0 / ((1 + MKT["tau"] * MKT["F0"][0]) * (1 + MKT["tau"] * MKT["F0"][1]))
    for steps in sorted({c["steps"] for c in GOLD["cases"]}):  # a batch shares its step count
        cases = [c for c in GOLD["cases"] if c["steps"] == steps]
        prices = B.solve_batch([caplet(c) for c in cases])
        for c, u in zip(cases, prices):
            bps = 1e4 * P2 * MKT["tau"] * u
            assert abs(bps - c["bps"]) <= 5.5e-7, (c["id"], bps, c["bps"])


def test_steps_resume_on_large_grids():
    inst = dict(W.c1_instance(), level=7, n_steps=8)
    a = B.Problem(inst)
    a.step(8)
    b = B.Problem(inst)
    b.step(3)
    b.step(5)
    assert abs(a.combine() - b.combine()) <= 1e-14 * max(1.0, abs(a.combine()))


def test_batch_mixing_small_and_large_grids():
    big = dict(W.c1_instance(), level=8, n_steps=4)
    insts = [W.c2_instance(3), big, W.small_instance(3, 9, steps=4, seed=9), W.c2_instance(4)]
    insts = [dict(x, n_steps=4) for x in insts]
    p = B.solve_batch(insts)
    for i, inst in enumerate(insts):
        pr = B.Problem(inst)
        pr.step(4)
        assert abs(pr.combine() - p[i]) <= TOL64 * abs(p[i]), i
        pr.close()
