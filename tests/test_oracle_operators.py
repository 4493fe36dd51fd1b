"""Pins of the oracle's spatial operator (Sketch 1), its directional splitting
(eqs. odeNd, ffis) and the line solves (Lemma ls, Algorithm 1).

- Consistency: on a smooth w with zero normal derivative and zero third
  normal derivative on the upper faces, F(w) at every Inner node converges at
  O(h^2) to L w, where L is the operator of the ORIGINAL form of the PDE,
  eq. (mmNd_no) of Sec. 2 (double sum over i, j with the factor 1/2, the drift
  mu_i with mu_1 = 0, time reversed).  The oracle is written from the other
  form, eq. (mmNd) with the coefficients of eqs. (coef_diff), (coef_mix),
  (coef_adv); agreement checks that rewrite term by term, the Neumann rows
  (ghost node, zero gradient, zero mixed term) and the central differences.
- Structure: F vanishes on Outer rows; F_i only couples J and J +- E_i; the
  dense matrix of F equals sum_i A_i + A_0 with A_0 free of any diagonal.
- Line solves: orc_line_solve equals a dense LU solve of (I - nu dt A_i) K = G
  with A_i assembled column by column from F_i (eq. ffis), and its residual is
  at rounding level.
"""
import math

import numpy as np
import pytest

import oracle as O


def inst_general(N, beta=0.5, sigma=0.35, seed=0):
    rng = np.random.default_rng(seed)
    nr = N - 1
    T = 0.5 * (1 + np.arange(nr))
    rho = np.exp(-0.3 * np.abs(T[:, None] - T[None, :]))
    return dict(N=N, payoff="swaption", n_steps=4, alpha=rng.uniform(0.15, 0.4, nr),
                phi=rng.uniform(-0.5, 0.3, nr), tau=rng.uniform(0.4, 0.6, nr),
                F0=rng.uniform(0.01, 0.03, nr), Fmax=rng.uniform(0.05, 0.2, nr), Vmax=2.5,
                rho=rho, sigma=sigma, beta=beta, V0=1.0, K=0.02, T=1.0,
                theta=(3 + math.sqrt(3)) / 6, nu=N * (3 + math.sqrt(3)) / 6, discount=1.0)


def coords(inst, levels):
    N = inst["N"]
    c = list(inst["Fmax"][: N - 1]) + [inst["Vmax"]]
    axes = [np.linspace(0.0, c[i], (1 << int(levels[i])) + 1) for i in range(N)]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    X = [m.ravel() for m in reversed(mesh)]  # axis-1-fastest flattening (theta_0)
    return X, c


def manufactured(X, c):
    """w = prod_i (1 + sin(pi x_i / (2 c_i))) and its derivatives."""
    N = len(X)
    k = [math.pi / (2 * c[i]) for i in range(N)]
    s = [1.0 + np.sin(k[i] * X[i]) for i in range(N)]
    ds = [k[i] * np.cos(k[i] * X[i]) for i in range(N)]
    dds = [-k[i] ** 2 * np.sin(k[i] * X[i]) for i in range(N)]

    def prod_except(skip, repl):
        v = np.ones_like(X[0])
        for i in range(N):
            v = v * (repl[i] if i in skip else s[i])
        return v

    w = prod_except(set(), {})
    w1 = [prod_except({i}, {i: ds[i]}) for i in range(N)]
    w2 = [[prod_except({i, j}, {i: ds[i], j: ds[j]}) if i != j else prod_except({i}, {i: dds[i]})
           for j in range(N)] for i in range(N)]
    return w, w1, w2


def L_mmNd_no(inst, X, w1, w2):
    """Operator of eq. (mmNd_no) (Sec. 2) acting on u, written from that form:
    1/2 s^2 V^2 u_VV + 1/2 V^2 sum_{i,j} a_i a_j rho_ij F_i^b F_j^b u_ij
    + s V^2 sum_i a_i phi_i F_i^b u_iV + sum_i mu_i F_i^b u_i,
    mu_1 = 0, mu_i = a_i V^2 sum_{j=2}^{i} tau_j F_j^b / (1 + tau_j F_j) rho_ij a_j.
    The time-to-maturity form has u_t = L u."""
    N = inst["N"]
    nr = N - 1
    V = X[N - 1]
    b = inst["beta"]
    al, ph, ta = np.asarray(inst["alpha"]), np.asarray(inst["phi"]), np.asarray(inst["tau"])
    rho = np.asarray(inst["rho"])
    sg = inst["sigma"]
    Fb = [X[i] ** b for i in range(nr)]
    out = 0.5 * sg * sg * V * V * w2[N - 1][N - 1]
    for i in range(nr):
        for j in range(nr):
            out = out + 0.5 * V * V * al[i] * al[j] * rho[i, j] * Fb[i] * Fb[j] * w2[i][j]
    for i in range(nr):
        out = out + sg * V * V * al[i] * ph[i] * Fb[i] * w2[i][N - 1]
    for i in range(1, nr):  # mu_1 = 0
        mu = np.zeros_like(V)
        for j in range(1, i + 1):
            mu = mu + ta[j] * Fb[j] / (1 + ta[j] * X[j]) * rho[i, j] * al[j]
        mu = al[i] * V * V * mu
        out = out + mu * Fb[i] * w1[i]
    return out


def inner_mask(levels):
    N = len(levels)
    axes = [np.arange((1 << int(l)) + 1) for l in levels]
    mesh = np.meshgrid(*reversed(axes), indexing="ij")
    J = [m.ravel() for m in reversed(mesh)]
    m = np.ones_like(J[0], dtype=bool)
    for i in range(N):
        m &= J[i] > 0
    return m


@pytest.mark.parametrize("N", [2, 3, 4])
def test_F_consistent_with_original_pde(N):
    inst = inst_general(N, seed=N)
    errs = []
    for lev in (2, 3, 4) if N <= 3 else (2, 3):
        levels = [lev] * N
        X, c = coords(inst, levels)
        w, w1, w2 = manufactured(X, c)
        Fw = O.apply_F(inst, levels, w)
        Lw = L_mmNd_no(inst, X, w1, w2)
        m = inner_mask(levels)
        assert np.all(Fw[~m] == 0.0)
        errs.append(np.max(np.abs(Fw[m] - Lw[m])))
    rates = [errs[k] / errs[k + 1] for k in range(len(errs) - 1)]
    assert min(rates) > 3.3, (errs, rates)  # second order: factor ~4 per level


def dense(op, n):
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = op(e)
    return A


@pytest.mark.parametrize("N,levels", [(2, [2, 3]), (3, [1, 2, 2]), (4, [1, 1, 2, 1])])
def test_splitting_structure(N, levels):
    inst = inst_general(N, seed=10 + N)
    n = O.grid_size(N, levels)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    inner = inner_mask(levels)
    assert np.all(A[~inner] == 0.0)
    E = [1]
    for l in levels[:-1]:
        E.append(E[-1] * ((1 << l) + 1))
    Asum = np.zeros_like(A)
    for i in range(N):
        Ai = dense(lambda v: O.apply_Fi(inst, levels, i, v), n)
        rows, cols = np.nonzero(Ai)
        assert np.all(np.isin(cols - rows, [-E[i], 0, E[i]]))
        Asum += Ai
    A0 = A - Asum
    # the mixed and advection part never touches the diagonal
    assert np.max(np.abs(np.diag(A0))) < 1e-9 * np.max(np.abs(A))


@pytest.mark.parametrize("N,levels", [(2, [3, 4]), (3, [2, 0, 2]), (4, [1, 2, 1, 2]), (3, [0, 0, 0])])
def test_line_solve_equals_dense_solve(N, levels):
    inst = inst_general(N, seed=20 + N)
    n = O.grid_size(N, levels)
    inner = inner_mask(levels)
    rng = np.random.default_rng(5)
    for axis in range(N):
        Ai = dense(lambda v: O.apply_Fi(inst, levels, axis, v), n)
        nu_dt = 0.37
        G = rng.standard_normal(n) * inner  # right-hand sides vanish on Outer rows
        K = O.line_solve(inst, levels, axis, nu_dt, G)
        Kd = np.linalg.solve(np.eye(n) - nu_dt * Ai, G)
        assert np.max(np.abs(K - Kd)) <= 1e-13 * max(1.0, np.max(np.abs(Kd)))
        res = K - nu_dt * O.apply_Fi(inst, levels, axis, K) - G
        assert np.max(np.abs(res)) <= 1e-12 * max(1.0, np.max(np.abs(G)))


# ---------------------------------------------------------- spatial order 2
def _caplet_on_nodes(sigma, phi, beta, alpha, steps=64):
    # strike K = 0.01 and spot F0 = 0.0125 are nodes of every grid of level
    # >= 4 on [0, 0.04] (the payoff kink sits on a node), V0 = 1 is a node on
    # [0, 2]; 64 steps of the third-order scheme leave the time error far
    # below the spatial one
    return dict(N=2, payoff="caplet", n_steps=steps, alpha=[alpha], phi=[phi], tau=[0.5],
                F0=[0.0125], Fmax=[0.04], Vmax=2.0, rho=[[1.0]], sigma=sigma, beta=beta, V0=1.0,
                K=0.01, T=0.5, theta=(3 + math.sqrt(3)) / 6, nu=(3 + math.sqrt(3)) / 6,
                discount=1.0)


def test_full_grid_price_converges_at_second_order_to_black():
    """Sec. 3 discretises with second-order central differences.  With sigma
    = 0 and beta = 1 the model is Black's lognormal one, whose caplet value
    (F N(d1) - K N(d2), volatility alpha V0) is exact; the error of the
    full-grid price falls by a factor tending to 4 per level (observed order
    2; the domain truncation at F^max, eight standard deviations away, is far
    below the errors measured here)."""
    F, K, vol, T = 0.0125, 0.01, 0.2, 0.5
    d1 = (math.log(F / K) + 0.5 * vol * vol * T) / (vol * math.sqrt(T))
    Nc = lambda x: 0.5 * (1.0 + math.erf(x / math.sqrt(2.0)))
    black = F * Nc(d1) - K * Nc(d1 - vol * math.sqrt(T))
    inst = _caplet_on_nodes(0.0, 0.0, 1.0, vol)
    err = [O.price(inst, lev, full=True) - black for lev in (6, 7, 8)]
    assert abs(err[2]) < 2e-5 * black  # 1.6e-5 relative at level 8 (257 x 257 nodes)
    r67, r78 = err[0] / err[1], err[1] / err[2]
    assert 3.0 < r67 < r78 < 4.3, (r67, r78)


def test_full_grid_self_convergence_with_stochastic_volatility():
    """The same on the SABR problem (sigma > 0, correlated, beta = 1/2),
    which has no closed form: the level-to-level price differences shrink by
    a factor that grows towards 4."""
    inst = _caplet_on_nodes(0.3, -0.3, 0.5, 0.02)
    p = [O.price(inst, lev, full=True) for lev in (5, 6, 7, 8)]
    d = [p[i] - p[i + 1] for i in range(3)]
    r1, r2 = d[0] / d[1], d[1] / d[2]
    assert 1.2 < r1 < r2 < 4.3 and r2 > 3.0, (r1, r2)
