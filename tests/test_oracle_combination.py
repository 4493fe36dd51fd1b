"""Pins of the oracle's grid enumeration, combination coefficients and
multilinear interpolation (Sec. 5, eqs. standardCombTechnique and
modifiedCombTechnique).

- the number of component grids is sum_q C(n-q+d-1, d-1) (Sec. 5.1);
- the coefficients sum to one;
- the union of the component grids has exactly the number of points the
  paper prints in Tables d2_1, d1:Level, sg_d3 and d4:level (this fixes the
  level convention: 2^l + 1 points on an axis of level l >= 0);
- the combined interpolant reproduces, to rounding, any function of the
  sparse space sum_{|l|=n} V_{psi 1 + l}: the combination technique applied to
  interpolation is the sparse-grid interpolation operator.  The test functions
  are built here with an independent numpy multilinear interpolator.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_tables.json")))


@pytest.mark.parametrize("d,n,psi", [(2, 6, 0), (3, 5, 0), (4, 5, 0), (6, 6, 1), (8, 4, 0), (5, 2, 0)])
def test_grid_count_and_coefficients(d, n, psi):
    lv, cf = O.enumerate_grids(d, n, psi)
    expect = sum(math.comb(n - q + d - 1, d - 1) for q in range(d) if n - q >= 0)
    assert len(lv) == expect
    # levels: psi + l with |l|_1 = n - q, coefficient (-1)^q C(d-1, q)
    for l, c in zip(lv, cf):
        q = n - int(np.sum(l - psi))
        assert 0 <= q < d and np.all(l >= psi)
        assert c == (-1) ** q * math.comb(d - 1, q)
    # no duplicates
    assert len({tuple(x) for x in lv}) == len(lv)
    if n >= d - 1:
        assert abs(cf.sum() - 1.0) < 1e-12


def test_full_grid_enumeration():
    lv, cf = O.enumerate_grids(3, 5, 0, full=True)
    assert lv.tolist() == [[5, 5, 5]] and cf.tolist() == [1.0]


def union_points(d, n, psi):
    lv, _ = O.enumerate_grids(d, n, psi)
    top = int(lv.max())
    pts = set()
    for l in lv:
        axes = [range(0, (1 << top) + 1, 1 << (top - int(li))) for li in l]
        pts.update(itertools.product(*axes))
    return len(pts)


@pytest.mark.parametrize("c", GOLD["point_counts"], ids=[c["source"] for c in GOLD["point_counts"]])
def test_union_point_counts_match_paper(c):
    if c["d"] >= 4:
        pytest.importorskip("numpy")  # always present; large case kept for completeness
    assert union_points(c["d"], c["n"], c["psi"]) == c["points"]


@pytest.mark.parametrize("c", GOLD["full_grid_points"], ids=[c["source"] for c in GOLD["full_grid_points"]])
def test_full_grid_point_counts_match_paper(c):
    assert O.grid_size(c["d"], [c["level"]] * c["d"]) == c["points"]


def _inst(d, cmax):
    nr = d - 1
    return dict(N=d, payoff="caplet", n_steps=1, alpha=[0.2] * nr, phi=[0.0] * nr,
                tau=[0.5] * nr, F0=[0.01] * nr, Fmax=list(cmax[:nr]), Vmax=cmax[nr],
                rho=np.eye(nr), sigma=0.0, beta=1.0, V0=1.0, K=0.0, T=1.0, theta=1.0,
                nu=1.0, discount=1.0)


def np_multilinear(values, levels, cmax, x):
    """Independent multilinear interpolation of a (M_1+1) x ... array (axis 1
    fastest in memory, i.e. values[j_d, ..., j_1] in C order)."""
    d = len(levels)
    idx, wts = [], []
    for i in range(d):
        M = 1 << int(levels[i])
        s = x[i] / cmax[i] * M
        c = min(int(math.floor(s)), M - 1)
        idx.append(c)
        wts.append(s - c)
    v = 0.0
    for corner in itertools.product((0, 1), repeat=d):
        w = 1.0
        for i in range(d):
            w *= wts[i] if corner[i] else 1.0 - wts[i]
        v += w * values[tuple(idx[i] + corner[i] for i in reversed(range(d)))]
    return v


def grid_nodes(levels, cmax):
    axes = [np.linspace(0.0, cmax[i], (1 << int(levels[i])) + 1) for i in range(len(levels))]
    # C-order array indexed [j_d, ..., j_1] so that axis 1 is fastest
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return [m for m in reversed(mesh)]  # coordinate arrays for axis 1..d


@pytest.mark.parametrize("d,n,psi", [(2, 4, 0), (3, 3, 0), (3, 2, 1), (4, 3, 0), (2, 3, 2)])
def test_combination_reproduces_sparse_space(d, n, psi):
    rng = np.random.default_rng(100 + 10 * d + n + psi)
    cmax = rng.uniform(0.5, 2.0, size=d)
    inst = _inst(d, cmax)
    # f = sum of random full-grid interpolants on the top-level grids |l| = n
    top = [l for l in itertools.product(range(n + 1), repeat=d) if sum(l) == n]
    parts = []
    for l in top:
        lv = np.array(l) + psi
        shape = tuple((1 << int(x)) + 1 for x in reversed(lv))
        parts.append((lv, rng.standard_normal(shape)))

    def f(x):
        return sum(np_multilinear(vals, lv, cmax, x) for lv, vals in parts)

    grids, coefs = O.enumerate_grids(d, n, psi)
    xs = rng.uniform(0.0, 1.0, size=(6, d)) * cmax
    for x in xs:
        tot = 0.0
        for lv, c in zip(grids, coefs):
            coords = grid_nodes(lv, cmax)
            vals = np.empty(coords[0].shape)
            for idx in np.ndindex(vals.shape):
                vals[idx] = f([coords[i][idx] for i in range(d)])
            tot += c * O.interp(inst, lv, vals.ravel(), list(x))
        assert abs(tot - f(x)) < 1e-11 * max(1.0, abs(f(x)))


def test_interp_is_exact_for_multilinear_and_at_nodes():
    rng = np.random.default_rng(7)
    d = 3
    cmax = np.array([0.2, 0.3, 1.5])
    inst = _inst(d, cmax)
    lv = np.array([2, 1, 3])
    coords = grid_nodes(lv, cmax)
    a = rng.standard_normal(8)

    def ml(x):  # a generic multilinear function
        v = 0.0
        for k, bits in enumerate(itertools.product((0, 1), repeat=3)):
            t = a[k]
            for i in range(3):
                if bits[i]:
                    t *= x[i]
            v += t
        return v

    vals = ml([coords[0], coords[1], coords[2]])
    for x in rng.uniform(0, 1, size=(10, 3)) * cmax:
        assert abs(O.interp(inst, lv, vals.ravel(), list(x)) - ml(x)) < 1e-13
    # at a node, and on the upper faces
    assert abs(O.interp(inst, lv, vals.ravel(), list(cmax)) - ml(cmax)) < 1e-13
    node = [coords[i][1, 1, 2] for i in range(3)]
    assert abs(O.interp(inst, lv, vals.ravel(), node) - vals[1, 1, 2]) < 1e-14


def test_modified_combination_converges_at_the_sparse_grid_rate():
    """Sec. 5 states the combination error as O(h^2 log(1/h)^(d-1)), i.e. a
    factor 4n/(n+1) per level for d = 2.  On the d=2 SABR caplet (payoff kink
    and spot on nodes, 64 steps) the level-to-level differences of the
    modified combination (psi = 1) shrink by factors growing towards that,
    and the level-9 combination approaches the level-8 full grid (to 2e-5
    relative, closer than the level-6 combination)."""
    theta = (3 + math.sqrt(3)) / 6
    inst = dict(N=2, payoff="caplet", n_steps=64, alpha=[0.02], phi=[-0.3], tau=[0.5],
                F0=[0.0125], Fmax=[0.04], Vmax=2.0, rho=[[1.0]], sigma=0.3, beta=0.5, V0=1.0,
                K=0.01, T=0.5, theta=theta, nu=theta, discount=1.0)
    p = [O.price(inst, lev, psi=1) for lev in (6, 7, 8, 9)]
    d = [p[i] - p[i + 1] for i in range(3)]
    r = [d[i] / d[i + 1] for i in range(2)]
    assert 2.0 < r[0] < r[1] < 4.0 and r[1] > 3.2, r
    full = O.price(inst, 8, full=True)  # 257 x 257 nodes
    assert abs(p[-1] - full) < 2e-5 * abs(full) and abs(p[-1] - full) < abs(p[0] - full), (p, full)
