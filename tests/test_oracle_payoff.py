"""Pin of the oracle's payoffs (Sec. 2).

The swaption payoff g is checked against the IRS value of eq. (swap) written
through zero-coupon bonds, IRS(T_a) = sum_{i=a}^{b-1} P(T_a, T_{i+1}) tau_i
(F_i - K) with P(T_i, T_j) = prod_{k=i}^{j-1} 1/(1 + tau_k F_k), a = 1, taken
positive part; the caplet payoff is (F_1 - K)^+.  Both are sampled on every
node of a small grid (Outer nodes included, they carry the Dirichlet data).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from test_oracle_operators import coords, inst_general


def bond(F, tau, i, j):
    p = 1.0
    for k in range(i, j):
        p = p / (1.0 + tau[k] * F[k])
    return p


@pytest.mark.parametrize("N", [2, 3, 5])
def test_swaption_payoff_is_positive_irs(N):
    inst = inst_general(N, seed=70 + N)
    inst["K"] = 0.05
    levels = [2] * N
    Y = O.payoff_grid(inst, levels)
    X, _ = coords(inst, levels)
    tau = np.asarray(inst["tau"])
    for J in range(Y.size):
        F = [X[i][J] for i in range(N - 1)]
        irs = sum(bond(F, tau, 0, i + 1) * tau[i] * (F[i] - inst["K"]) for i in range(N - 1))
        assert abs(Y[J] - max(irs, 0.0)) < 1e-15


def test_caplet_payoff():
    inst = dict(inst_general(3, seed=3), payoff="caplet", K=0.04)
    levels = [3, 1, 1]
    Y = O.payoff_grid(inst, levels)
    X, _ = coords(inst, levels)
    assert np.array_equal(Y, np.maximum(X[0] - 0.04, 0.0))
