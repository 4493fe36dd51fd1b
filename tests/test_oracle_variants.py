"""Pins of the oracle's method variants (the paper's comparisons, not the hot
path): the theta-method with Gauss-Seidel iterations read as a W-method
(Sec. 4.2, eqs. thetamet and GS), the earlier Dirichlet boundary conditions of
eq. bound1_0 (Sec. 2), and the AMF parameter nu.

theta-method + Gauss-Seidel, s iterations per step (W = P, the lower triangle
of A with its diagonal; a_rj = theta, q_rj = -1, b_r = 1):
- with many iterations one step converges to the theta-method step
  (I - theta dt A) W_1 = (I + (1 - theta) dt A) W_0 solved by dense LU;
- two iterations equal the W-method written densely with numpy's triangle;
- order against expm(T A): 2 for theta = 1/2 with s = 2, 1 for theta = 1 or
  for a single iteration (Sec. 4.2 states order 2 only for theta = 1/2,
  s >= 2).

Dirichlet conditions of eq. bound1_0 (u = g on every face F_j = F_j^max; V
keeps dU/dV = 0 at V^max):
- any grid function linear in the rates is reproduced exactly (its second
  differences vanish and the boundary data are exact), while the Neumann
  ghost node of Sketch 1 bends it at the upper face;
- F is second-order consistent with the operator of eq. mmNd_no on the new
  Inner set; the line solves equal dense LU; one AMFR-W2 step equals the
  dense W-method of eqs. row-s/Wmat1; the order at theta* stays 3;
- the caplet of Sec. 6.1 converges to Black's price as with Sketch 1.

nu: the AMFR-W2 order 3 at theta* holds for every nu (condition Wmfp does not
involve nu, Sec. 4.1).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from test_oracle_operators import L_mmNd_no, coords, dense, inst_general, manufactured

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_tables.json")))
THETA = (3 + math.sqrt(3)) / 6


def multi_index(levels):
    axes = [np.arange((1 << int(l)) + 1) for l in levels]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    return [m.ravel() for m in reversed(mesh)]  # axis-1-fastest (theta_0)


def inner(levels, bc="neumann"):
    J = multi_index(levels)
    N = len(levels)
    m = np.ones_like(J[0], dtype=bool)
    for i in range(N):
        m &= J[i] > 0
        if bc == "dirichlet" and i < N - 1:
            m &= J[i] < (1 << int(levels[i]))
    return m


def start(inst, levels, seed, bc="neumann"):
    """Outer nodes carry the payoff, Inner nodes a smooth random surface."""
    Y = O.payoff_grid(inst, levels)
    rng = np.random.default_rng(seed)
    n = Y.size
    m = inner(levels, bc)
    t = np.linspace(0, 1, n)
    Y[m] = (0.01 + 0.02 * np.sin(3 * t) + 1e-4 * rng.standard_normal(n))[m]
    return Y


def slopes(errs):
    e = np.asarray(errs)
    return np.log2(e[:-1] / e[1:])


# ------------------------------------------------------ theta + Gauss-Seidel
def test_theta_gs_converges_to_theta_method():
    N, levels = 2, [2, 2]
    for theta in (0.5, 1.0):
        inst = dict(inst_general(N, seed=61), theta=theta, T=0.05, n_steps=4)
        dt = inst["T"] / inst["n_steps"]
        n = O.grid_size(N, levels)
        A = dense(lambda v: O.apply_F(inst, levels, v), n)
        Y0 = start(inst, levels, 3)
        W1 = np.linalg.solve(np.eye(n) - theta * dt * A, (np.eye(n) + (1 - theta) * dt * A) @ Y0)
        Y1 = O.run_theta_gs(inst, levels, Y0, s_iter=60, n_steps=1)
        assert np.max(np.abs(Y1 - W1)) <= 1e-13 * np.max(np.abs(W1)), theta


@pytest.mark.parametrize("N,levels", [(2, [2, 3]), (3, [1, 2, 1])])
def test_theta_gs_two_iterations_equal_dense_W_method(N, levels):
    inst = dict(inst_general(N, seed=70 + N), theta=0.5)
    dt = inst["T"] / inst["n_steps"]
    n = O.grid_size(N, levels)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    M = np.eye(n) - 0.5 * dt * np.tril(A)
    Y0 = O.payoff_grid(inst, levels)
    K1 = np.linalg.solve(M, dt * A @ Y0)
    K2 = np.linalg.solve(M, dt * A @ (Y0 + 0.5 * K1) - K1)
    Y1 = Y0 + K1 + K2
    Yo = O.run_theta_gs(inst, levels, Y0, s_iter=2, n_steps=1)
    assert np.max(np.abs(Yo - Y1)) <= 1e-13 * max(1.0, np.max(np.abs(Y1)))


@pytest.mark.parametrize("theta,s_iter,order", [(0.5, 2, 2), (0.5, 3, 2), (1.0, 2, 1), (0.5, 1, 1)])
def test_theta_gs_order(theta, s_iter, order):
    N, levels = 2, [2, 2]
    inst = dict(inst_general(N, seed=81), T=0.25, theta=theta)
    n = O.grid_size(N, levels)
    Y0 = start(inst, levels, 4)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Yex = sla.expm(inst["T"] * A) @ Y0
    errs = []
    for steps in (32, 64, 128, 256):
        Y = O.run_theta_gs(dict(inst, n_steps=steps), levels, Y0, s_iter=s_iter)
        errs.append(np.max(np.abs(Y - Yex)))
    sl = slopes(errs)
    assert abs(sl[-1] - order) < 0.25 and abs(sl[-2] - order) < 0.35, (errs, sl)


def test_theta_gs_rejects_large_grids():
    inst = inst_general(2, seed=1)
    with pytest.raises(ValueError):
        O.run_theta_gs(inst, [6, 6], O.payoff_grid(inst, [6, 6]), s_iter=1)


# ------------------------------------------------- Dirichlet, eq. bound1_0
@pytest.mark.parametrize("N,levels", [(2, [3, 3]), (3, [2, 2, 2]), (4, [2, 1, 1, 2])])
def test_dirichlet_reproduces_solutions_linear_in_the_rates(N, levels):
    # caplet with K = 0: g = F_1 on F_1 >= 0 solves the PDE (every derivative
    # the operator takes of it vanishes), and so does its grid restriction
    base = dict(inst_general(N, seed=90 + N), payoff="caplet", K=0.0, n_steps=6)
    g = O.payoff_grid(base, levels)
    Yd = O.run(dict(base, bc="dirichlet"), levels, g)
    assert np.max(np.abs(Yd - g)) <= 1e-15 * np.max(np.abs(g)) * 100
    Yn = O.run(base, levels, g)
    J = multi_index(levels)
    top = J[0] == (1 << levels[0])
    dev = np.abs(Yn - g)
    assert dev[top & inner(levels)].max() > 1e-6 * np.max(np.abs(g))
    assert dev[~top].max() < dev[top].max()


@pytest.mark.parametrize("N", [2, 3, 4])
def test_dirichlet_F_consistent_with_original_pde(N):
    inst = dict(inst_general(N, seed=N), bc="dirichlet")
    errs = []
    for lev in (3, 4, 5) if N <= 3 else (3, 4):
        levels = [lev] * N
        X, c = coords(inst, levels)
        w, w1, w2 = manufactured(X, c)
        Fw = O.apply_F(inst, levels, w)
        Lw = L_mmNd_no(inst, X, w1, w2)
        m = inner(levels, "dirichlet")
        assert np.all(Fw[~m] == 0.0)
        errs.append(np.max(np.abs(Fw[m] - Lw[m])))
    rates = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    # second order: the error ratio per level approaches 4 (N = 3: 2.53, 3.48,
    # 3.80 from level 2 on; N = 4: 2.53, 3.23)
    assert rates[-1] > 3.2 and min(rates) > 3.0, (errs, rates)


@pytest.mark.parametrize("N,levels", [(2, [3, 4]), (3, [2, 1, 2]), (4, [1, 2, 2, 2]), (3, [1, 1, 1])])
def test_dirichlet_line_solve_equals_dense_solve(N, levels):
    inst = dict(inst_general(N, seed=20 + N), bc="dirichlet")
    n = O.grid_size(N, levels)
    m = inner(levels, "dirichlet")
    rng = np.random.default_rng(6)
    for axis in range(N):
        Ai = dense(lambda v: O.apply_Fi(inst, levels, axis, v), n)
        assert np.all(Ai[~m] == 0.0)
        G = rng.standard_normal(n) * m
        K = O.line_solve(inst, levels, axis, 0.41, G)
        Kd = np.linalg.solve(np.eye(n) - 0.41 * Ai, G)
        assert np.max(np.abs(K - Kd)) <= 1e-13 * max(1.0, np.max(np.abs(Kd)))


@pytest.mark.parametrize("N,levels", [(2, [2, 3]), (3, [2, 1, 2])])
def test_dirichlet_one_step_equals_dense_W_method(N, levels):
    inst = dict(inst_general(N, seed=50 + N), bc="dirichlet")
    dt = inst["T"] / inst["n_steps"]
    th, nu = inst["theta"], inst["nu"]
    n = O.grid_size(N, levels)
    I = np.eye(n)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Pinv = I.copy()
    for i in range(N):
        Ai = dense(lambda v: O.apply_Fi(inst, levels, i, v), n)
        Pinv = np.linalg.solve(I - nu * dt * Ai, Pinv)
    Winv = Pinv @ (2 * I - (I - th * dt * A) @ Pinv)
    Y0 = O.payoff_grid(inst, levels)
    K1 = Winv @ (dt * A @ Y0)
    K2 = Winv @ (dt * A @ (Y0 + 2.0 / 3.0 * K1) - 4.0 / 3.0 * K1)
    Y1 = Y0 + 1.25 * K1 + 0.75 * K2
    Yo = O.run(inst, levels, Y0, n_steps=1)
    assert np.max(np.abs(Yo - Y1)) <= 1e-13 * max(1.0, np.max(np.abs(Y1)))


def test_dirichlet_order_three_at_theta_star():
    N, levels = 2, [2, 3]
    inst = dict(inst_general(N, seed=33), T=0.25, bc="dirichlet")
    n = O.grid_size(N, levels)
    Y0 = start(inst, levels, 5, "dirichlet")
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Yex = sla.expm(inst["T"] * A) @ Y0
    errs = [np.max(np.abs(O.run(dict(inst, n_steps=s), levels, Y0) - Yex)) for s in (16, 32, 64, 128)]
    sl = slopes(errs)
    assert sl[-1] > 2.7 and sl[-2] > 2.6, (errs, sl)


def test_dirichlet_caplet_converges_to_black():
    # Sec. 6.1: beta = 1, sigma = 0 is Black's model; the printed Black price
    mkt = GOLD["market"]
    black = GOLD["black_caplet_bps"]["value"]
    P2 = 1.0 / ((1 + mkt["tau"] * mkt["F0"][0]) * (1 + mkt["tau"] * mkt["F0"][1]))
    inst = dict(N=2, payoff="caplet", n_steps=16, alpha=[mkt["alpha"][1]], phi=[0.0],
                tau=[mkt["tau"]], F0=[mkt["F0"][1]], Fmax=[mkt["Fmax"]], Vmax=mkt["Vmax"],
                rho=[[1.0]], sigma=0.0, beta=1.0, V0=mkt["V0"], K=mkt["K"], T=mkt["T"][1],
                theta=THETA, nu=THETA, discount=1.0)
    err = {}
    for bc in ("neumann", "dirichlet"):
        for lev in (5, 6, 7):
            u = O.price(dict(inst, bc=bc), lev, full=True)
            err[bc, lev] = abs(1e4 * P2 * mkt["tau"] * u - black)
    for bc in ("neumann", "dirichlet"):
        assert err[bc, 7] < err[bc, 6] < err[bc, 5], err
        assert err[bc, 7] < 5e-3 * black, err
    # the caplet expires far from F^max: both conditions give the same price
    assert abs(err["dirichlet", 7] - err["neumann", 7]) < 1e-3 * black, err


# ------------------------------------------------------------------ nu sweep
@pytest.mark.parametrize("nu_factor", [0.5, 1.0, 2.0])
def test_amfrw2_order_three_for_every_nu(nu_factor):
    N, levels = 2, [2, 2]
    inst = dict(inst_general(N, seed=34), T=0.25, theta=THETA, nu=nu_factor * N * THETA)
    n = O.grid_size(N, levels)
    Y0 = start(inst, levels, 7)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Yex = sla.expm(inst["T"] * A) @ Y0
    errs = [np.max(np.abs(O.run(dict(inst, n_steps=s), levels, Y0) - Yex)) for s in (16, 32, 64, 128)]
    sl = slopes(errs)
    assert sl[-1] > 2.7 and sl[-2] > 2.6, (nu_factor, errs, sl)
