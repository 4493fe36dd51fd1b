"""Pin of the CPU reference network (oracle/mlp.py): its analytic gradients
equal central finite differences of its own loss, parameter by parameter,
on a small network in FP64; and gelu' equals the finite difference of gelu."""
import numpy as np

from oracle import mlp


def test_gelu_grad_is_derivative():
    z = np.linspace(-4, 4, 41)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(z))) < 1e-8


def test_gradients_match_finite_differences():
    p = mlp.init_params(width=12, n_in=8, seed=3)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, size=(9, 8))
    t = rng.standard_normal(9)
    _, g = mlp.loss_and_grads(p, X, t)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        val = np.array(p[name], dtype=np.float64)
        flat = val.reshape(-1)
        gflat = np.array(g[name], dtype=np.float64).reshape(-1)
        for k in range(0, flat.size, max(1, flat.size // 7)):
            save = flat[k]
            flat[k] = save + h
            p[name] = flat.reshape(val.shape) if val.ndim else float(flat[0])
            lp, _ = mlp.loss_and_grads(p, X, t)
            flat[k] = save - h
            p[name] = flat.reshape(val.shape) if val.ndim else float(flat[0])
            lm, _ = mlp.loss_and_grads(p, X, t)
            flat[k] = save
            p[name] = flat.reshape(val.shape) if val.ndim else float(flat[0])
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gflat[k]) <= 1e-7 * max(1.0, abs(fd)), (name, k, fd, gflat[k])


def test_grad_abs_scale_bounds_every_gradient_entry():
    # |sum_b a_b c_b| <= sum_b |a_b| |c_b| at every step of the chain rule,
    # and with every factor positive (inputs, weights, residuals, GELU
    # derivatives) the two coincide
    p = mlp.init_params(width=16, n_in=8, seed=2)
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(32, 8))
    t = rng.standard_normal(32)
    _, g = mlp.loss_and_grads(p, x, t)
    s = mlp.grad_abs_scale(p, x, t)
    for name in g:
        assert np.all(np.abs(g[name]) <= np.asarray(s[name]) * (1 + 1e-12) + 1e-300), name
    q = {k: (np.abs(v) if isinstance(v, np.ndarray) else abs(v)) for k, v in p.items()}
    xp = np.abs(x)
    tp = np.full(32, -100.0)
    _, g = mlp.loss_and_grads(q, xp, tp)
    s = mlp.grad_abs_scale(q, xp, tp)
    for name in g:
        assert np.allclose(np.abs(g[name]), s[name], rtol=1e-12, atol=0), name
