"""Plain FP64 CPU reference of the surrogate network (test infrastructure).

The network maps 8 normalised features to a normalised price:
    Z1 = X W1^T + b1, H1 = gelu(Z1)        (W1: 256 x 8)
    Z2 = H1 W2^T + b2, H2 = gelu(Z2)       (W2: 256 x 256)
    Z3 = H2 W3^T + b3, H3 = gelu(Z3)       (W3: 256 x 256)
    y  = H3 w4 + b4                        (w4: 256)
with gelu(z) = z Phi(z) (Phi the standard normal CDF) and the loss
L = 1/2 mean_b (y_b - t_b)^2.  Gradients by the chain rule, written out
layer by layer.  Only tests/ use this module; the CUDA library never does.
Pinned by tests/test_oracle_mlp.py against central finite differences.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def forward(p: dict, X: np.ndarray):
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = gelu(Z2)
    Z3 = H2 @ p["W3"].T + p["b3"]
    H3 = gelu(Z3)
    y = H3 @ p["w4"] + p["b4"]
    return y, (X, Z1, H1, Z2, H2, Z3, H3)


def loss_and_grads(p: dict, X: np.ndarray, t: np.ndarray):
    y, (X, Z1, H1, Z2, H2, Z3, H3) = forward(p, X)
    B = X.shape[0]
    r = y - t
    L = 0.5 * float(np.mean(r * r))
    dy = r / B
    g = {}
    g["w4"] = H3.T @ dy
    g["b4"] = np.sum(dy)
    dZ3 = np.outer(dy, p["w4"]) * gelu_grad(Z3)
    g["W3"] = dZ3.T @ H2
    g["b3"] = dZ3.sum(axis=0)
    dZ2 = (dZ3 @ p["W3"]) * gelu_grad(Z2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * gelu_grad(Z1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return L, g


def grad_abs_scale(p: dict, X: np.ndarray, t: np.ndarray) -> dict:
    """Per-entry scale of every gradient: the chain rule of loss_and_grads
    with every factor replaced by its absolute value, e.g. for W3 the
    entries of |dZ3|^T |H2| with |dZ3| = |dy w4^T| |gelu'(Z3)|.  A gradient
    computed from rounded operands (BF16 weights and activations, relative
    rounding u = 2^-8) differs from the exact one by at most a small multiple
    of u times this scale, entry by entry, whatever the cancellation in the
    exact sum."""
    y, (X, Z1, H1, Z2, H2, Z3, H3) = forward(p, X)
    B = X.shape[0]
    ady = np.abs(y - t) / B
    s = {}
    s["w4"] = np.abs(H3).T @ ady
    s["b4"] = float(np.sum(ady))
    a3 = np.outer(ady, np.abs(p["w4"])) * np.abs(gelu_grad(Z3))
    s["W3"] = a3.T @ np.abs(H2)
    s["b3"] = a3.sum(axis=0)
    a2 = (a3 @ np.abs(p["W3"])) * np.abs(gelu_grad(Z2))
    s["W2"] = a2.T @ np.abs(H1)
    s["b2"] = a2.sum(axis=0)
    a1 = (a2 @ np.abs(p["W2"])) * np.abs(gelu_grad(Z1))
    s["W1"] = a1.T @ np.abs(X)
    s["b1"] = a1.sum(axis=0)
    return s


def init_params(width: int = 256, n_in: int = 8, seed: int = 0) -> dict:
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((width, n_in)) * math.sqrt(2.0 / n_in),
        "b1": rng.standard_normal(width) * 0.1,
        "W2": rng.standard_normal((width, width)) * math.sqrt(2.0 / width),
        "b2": rng.standard_normal(width) * 0.1,
        "W3": rng.standard_normal((width, width)) * math.sqrt(2.0 / width),
        "b3": rng.standard_normal(width) * 0.1,
        "w4": rng.standard_normal(width) * math.sqrt(1.0 / width),
        "b4": float(rng.standard_normal() * 0.1),
    }
