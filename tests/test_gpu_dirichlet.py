"""GPU parity of the earlier boundary conditions (eq. bound1_0, flag
AMFRW_FLAG_DIRICHLET) against the oracle's bc = 1 path, which
tests/test_oracle_variants.py pins (exact reproduction of rate-linear
solutions, O(h^2) consistency, dense LU, dense W-method, order 3, Black).

Under eq. bound1_0 the upper face of every rate axis holds the payoff as
Dirichlet data; the V axis keeps its Neumann face at V^max.  The GPU stores
those face nodes (Z = 0 there) and gives their rows of the directional
matrices the identity.  Every work-group kind is covered: warp groups (FP64
difference-array stencil, mixed table-driven stencil), whole-block groups in
shared memory and in global memory; prices and, node by node, sampled grids.
"""
import numpy as np
import pytest

import oracle as O
from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


def inner(Y_full, levels):
    shape = tuple((1 << int(l)) + 1 for l in reversed(levels))
    return Y_full.reshape(shape)[(slice(1, None),) * len(levels)].ravel()


CASES = [
    # (N, level, psi, full, precision, global grids, payoff)
    (2, 5, 0, True, "fp64", False, "caplet"),     # full grid, whole-block group
    (4, 3, 0, False, "fp64", False, "swaption"),  # warp groups, difference-array stencil
    (4, 3, 0, False, "mixed", False, "swaption"),  # warp groups, table-driven stencil
    (3, 4, 1, False, "fp64", True, "swaption"),   # global-memory groups
    (6, 2, 1, False, "mixed", False, "swaption"),
    (8, 3, 0, False, "mixed", False, "swaption"),
    (4, 7, 0, False, "fp64", False, "swaption"),  # grids beyond 64 nodes: whole-block groups
    (4, 7, 0, False, "mixed", False, "swaption"),  # the same in mixed precision (Z in the block's global slice)
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[0]}_n{c[1]}_psi{c[2]}{'_full' if c[3] else ''}_{c[4]}"
                                             f"{'_global' if c[5] else ''}" for c in CASES])
def test_dirichlet_price_and_grids_match_oracle(case):
    N, n, psi, full, prec, glob, payoff = case
    inst = W.small_instance(N, n, psi=psi, steps=6, seed=700 + N, precision=prec, full=full, payoff=payoff)
    inst = dict(inst, bc="dirichlet", global_grids=glob)
    tol = TOL64 if prec == "fp64" else TOLMIX
    prob = B.Problem(inst)
    prob.step(inst["n_steps"])
    p = prob.combine()
    po = O.price(inst, n, psi, full)
    assert abs(p - po) <= tol * abs(po), (p, po, abs(p - po) / abs(po))
    lv, _ = prob.grid_info()
    tol_grid = TOL64 if prec == "fp64" else 1e-6
    for g in sorted({0, len(lv) // 2, len(lv) - 1}):
        Yo = inner(O.solve_grid(inst, lv[g], want_Y=True)[1], lv[g])
        Yg = prob.read_grid(g, lv[g])
        scale = max(np.max(np.abs(Yo)), 1e-300)
        assert np.max(np.abs(Yg - Yo)) <= tol_grid * scale, (lv[g], np.max(np.abs(Yg - Yo)) / scale)
    prob.close()
    # the boundary condition changes the price (the Neumann problem differs)
    pn = O.price(dict(inst, bc="neumann"), n, psi, full)
    assert pn != po


def test_dirichlet_batch_matches_single_problems():
    insts = [dict(x, bc="dirichlet", n_steps=6) for x in W.batch("c4", 12, start=90, precision="fp64")]
    p = B.solve_batch(insts)
    for i in (0, 5, 11):
        pr = B.Problem(insts[i])
        pr.step(insts[i]["n_steps"])
        q = pr.combine()
        pr.close()
        assert abs(q - p[i]) <= 1e-12 * abs(q), (i, q, p[i])
