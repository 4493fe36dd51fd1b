"""Pins of the oracle's time integration (Sec. 4, eqs. row-s, Wmat1, amfrw,
coef_W2).

- Order: on tiny grids the semi-discrete system Y' = A Y (Outer rows of A are
  zero) has the exact solution expm(T A) Y0 (scipy's Pade expm, a library
  primitive).  The AMFR-W2 error must fall like dt^3 for
  theta = (3 + sqrt 3)/6 and like dt^2 for another theta (Sec. 4.1: the method
  has order 3 in the ODE sense only for that theta).
- Structure: one oracle step equals the W-method of eq. (row-s) written
  densely with (I - theta dt W)^{-1} from eq. (Wmat1),
  P^{-1} (2 I - (I - theta dt A) P^{-1}), P^{-1} = prod_{i=N}^{1} (I - nu dt A_i)^{-1},
  with the dense matrices assembled column by column from F and F_i.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from test_oracle_operators import dense, inner_mask, inst_general

THETA = (3 + math.sqrt(3)) / 6


def smooth_start(inst, levels, seed):
    """Outer nodes carry the payoff, Inner nodes a smooth random surface."""
    Y = O.payoff_grid(inst, levels)
    rng = np.random.default_rng(seed)
    n = Y.size
    inner = inner_mask(levels)
    t = np.linspace(0, 1, n)
    Y[inner] = (0.01 + 0.02 * np.sin(3 * t) + 0.005 * rng.standard_normal(n) * 0.01)[inner]
    return Y


def errors(inst, levels, steps_list, Y0):
    n = Y0.size
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Yex = sla.expm(inst["T"] * A) @ Y0
    out = []
    for s in steps_list:
        ii = dict(inst, n_steps=s)
        out.append(np.max(np.abs(O.run(ii, levels, Y0) - Yex)))
    return np.array(out)


@pytest.mark.parametrize("N,levels", [(2, [2, 2]), (3, [1, 2, 1])])
def test_order_three_at_theta_star(N, levels):
    inst = dict(inst_general(N, seed=30 + N), T=0.25, theta=THETA, nu=N * THETA)
    Y0 = smooth_start(inst, levels, 1)
    e = errors(inst, levels, [16, 32, 64, 128], Y0)
    slopes = np.log2(e[:-1] / e[1:])
    assert slopes[-1] > 2.7 and slopes[-2] > 2.6, (e, slopes)


@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_order_two_off_theta_star(theta):
    N, levels = 2, [2, 2]
    inst = dict(inst_general(N, seed=41), T=0.25, theta=theta, nu=N * theta)
    Y0 = smooth_start(inst, levels, 2)
    e = errors(inst, levels, [16, 32, 64, 128], Y0)
    slopes = np.log2(e[:-1] / e[1:])
    assert 1.7 < slopes[-1] < 2.3, (e, slopes)


@pytest.mark.parametrize("N,levels", [(2, [2, 3]), (3, [1, 2, 1]), (4, [1, 1, 1, 2])])
def test_one_step_equals_dense_W_method(N, levels):
    inst = inst_general(N, seed=50 + N)
    dt = inst["T"] / inst["n_steps"]
    th, nu = inst["theta"], inst["nu"]
    n = O.grid_size(N, levels)
    I = np.eye(n)
    A = dense(lambda v: O.apply_F(inst, levels, v), n)
    Pinv = I.copy()
    for i in range(N):  # prod_{i=N}^{1}: the i = 1 factor acts first
        Ai = dense(lambda v: O.apply_Fi(inst, levels, i, v), n)
        Pinv = np.linalg.solve(I - nu * dt * Ai, Pinv)
    Winv = Pinv @ (2 * I - (I - th * dt * A) @ Pinv)
    Y0 = O.payoff_grid(inst, levels)
    K1 = Winv @ (dt * A @ Y0)
    K2 = Winv @ (dt * A @ (Y0 + 2.0 / 3.0 * K1) - 4.0 / 3.0 * K1)
    Y1 = Y0 + 1.25 * K1 + 0.75 * K2
    Yo = O.run(inst, levels, Y0, n_steps=1)
    assert np.max(np.abs(Yo - Y1)) <= 1e-13 * max(1.0, np.max(np.abs(Y1)))
