"""GPU tests of the surrogate (ensemble MLP on the tensor cores, trained on
solver prices, solver fallback):

- the loss gradient computed by the network's forward/backward kernels
  (tcgen05 GEMMs with BF16 weights and activations, FP32 accumulation)
  agrees with the plain FP64 CPU reference (oracle/mlp.py, itself pinned by
  finite differences) entry by entry, every bias and padded input included:
  each entry within 16 BF16 roundoffs of the chain rule's absolute-value
  scale for that entry, and every tensor within 3 % relative L2 error with
  cosine similarity > 0.999;
- training (cubic control variate plus networks on the residual of the log
  price) drives the loss down; calibration and evaluation on fresh
  instances of the family give, for every answer the network keeps, an error
  within the bound in the calibrated fraction of cases, and answers that fall
  back are exactly the solver's prices; queries outside the family or the
  trained feature box always fall back;
- the same queries given as raw features get identical answers, faster than
  the solver alone prices them (the gain the network brings);
- save/load round-trips.
"""
import numpy as np
import pytest

from oracle import mlp
from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


def to_vector(p):
    lay = B.surrogate_layout()
    v = np.zeros(B.SURROGATE_PARAMS, dtype=np.float32)
    W1 = np.zeros((256, 16))
    W1[:, :8] = p["W1"]
    for name, arr in (("W1", W1), ("b1", p["b1"]), ("W2", p["W2"]), ("b2", p["b2"]), ("W3", p["W3"]),
                      ("b3", p["b3"]), ("w4", p["w4"]), ("b4", np.array([p["b4"]]))):
        o, n = lay[name]
        v[o:o + n] = np.asarray(arr, dtype=np.float64).reshape(-1)
    return v


def from_vector(g):
    lay = B.surrogate_layout()
    out = {}
    for name, shape in (("W1", (256, 16)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)),
                        ("W3", (256, 256)), ("b3", (256,)), ("w4", (256,)), ("b4", (1,))):
        o, n = lay[name]
        out[name] = g[o:o + n].astype(np.float64).reshape(shape)
    out["W1"] = out["W1"][:, :8]
    return out


# BF16 unit roundoff and the multiple of it, times the per-entry scale of the
# chain rule in absolute values, that bounds each gradient entry's error:
# each GEMM rounds both operands (2u), and the error reaches the first layer's
# gradient through three layers forward and back.
BF16_U = 2.0 ** -8
GRAD_K = 16.0


def test_gradients_match_cpu_oracle():
    s = B.Surrogate(members=1, seed=1)
    p = mlp.init_params(width=256, n_in=8, seed=5)
    v = to_vector(p)
    s.params(0, v)
    back = s.params(0)
    assert np.array_equal(back, v)
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, size=(256, 8))
    t = rng.standard_normal(256)
    g_gpu, loss_gpu = s.grad(0, x, t)
    # the reference uses the FP32 parameters the GPU holds
    p32 = from_vector(v)
    p32["b4"] = float(p32["b4"][0])
    L, g = mlp.loss_and_grads(p32, x, t)
    assert abs(loss_gpu - L) <= 1e-2 * L
    scale = mlp.grad_abs_scale(p32, x, t)
    lay = B.surrogate_layout()
    # the padded inputs 8..15 of the first layer carry no gradient at all
    o, n = lay["W1"]
    assert np.all(g_gpu[o:o + n].reshape(256, 16)[:, 8:] == 0.0)
    gg = from_vector(g_gpu)
    gg["b4"] = float(gg["b4"][0])
    worst = {}
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"):
        a = np.ravel(gg[name])
        b = np.ravel(g[name])
        sc = np.ravel(scale[name])
        # every entry, biases and b4 included, within its BF16 bound
        ratio = np.abs(a - b) / (BF16_U * sc + 1e-300)
        worst[name] = float(ratio.max())
        assert np.all(ratio <= GRAD_K), (name, int(ratio.argmax()), worst[name])
        # and the tensor as a whole close to the reference
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        cos = float(np.dot(a, b) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-300))
        assert rel < 3e-2 and cos > 0.999, (name, rel, cos)
    print("gradient error / (u * scale), worst entry per tensor:", worst)
    s.close()


FAMILY = dict(N=4, level=5, steps=8)


def family(count, start):
    F = W.c5_features(count, start, N=FAMILY["N"])
    return F, [W.c5_instance_from(f, **FAMILY) for f in F]


def test_train_calibrate_eval_with_fallback(tmp_path):
    import time
    import torch
    (_, train), (_, audit), (F_test, test) = family(32768, 0), family(4096, 10_000), family(8192, 20_000)
    y_train = B.solve_batch(train)
    y_audit = B.solve_batch(audit)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    y_test = B.solve_batch(test)
    t_solver = time.perf_counter() - t0
    assert (y_train > 0).all()
    s = B.Surrogate(members=4, seed=7)
    loss = s.fit(train, y_train, epochs=300, lr=3e-3)
    assert loss < 1e-3, loss  # standardised residual targets start near 0.5
    c = s.calibrate(audit, y_audit, rel_bound=1e-3, quantile=0.99)
    assert c > 0
    prices, fell = s.eval(test)
    kept = ~fell
    rel = np.abs(prices - y_test) / np.abs(y_test)
    assert np.array_equal(prices[fell], y_test[fell])
    assert kept.mean() >= 0.5, kept.mean()
    assert np.mean(rel[kept] <= 1e-3) >= 0.98, np.mean(rel[kept] <= 1e-3)
    # the same queries as raw features: identical answers, and the gain over
    # the solver alone
    t0 = time.perf_counter()
    p_f, fell_f = s.eval_features(F_test)
    t_sur = time.perf_counter() - t0
    assert np.array_equal(p_f, prices) and np.array_equal(fell_f, fell)
    assert t_sur < t_solver, (t_sur, t_solver)
    # outside the family (another level) and outside the feature box (strike)
    odd = [dict(test[0], level=4), dict(test[1], K=0.031)]
    p_odd, f_odd = s.eval(odd)
    assert f_odd.all()
    assert np.allclose(p_odd, B.solve_batch(odd), rtol=0, atol=0)
    # save / load
    path = tmp_path / "sg.bin"
    s.save(str(path))
    s2 = B.Surrogate.load(str(path))
    m1, sp1, _ = s.predict(test[:64])
    m2, sp2, _ = s2.predict(test[:64])
    assert np.array_equal(m1, m2) and np.array_equal(sp1, sp2)
    print(f"surrogate: loss {loss:.2e} calib {c:.2f} kept {kept.mean():.3f} "
          f"kept within 1e-3 {np.mean(rel[kept] <= 1e-3):.4f} max rel err kept {rel[kept].max():.2e} "
          f"median {np.median(rel[kept]):.2e}; {len(test)} queries: solver {t_solver:.3f} s, "
          f"surrogate+fallback {t_sur:.3f} s ({t_solver / t_sur:.1f}x)")


def test_lattice_feature_answers_only_on_its_values():
    # strikes on a lattice of 9 values: the network is trained and answers
    # there only; a strike between two lattice values falls back to the
    # solver (its price is not smooth in K between kinks of the payoff)
    kw = dict(N=4, level=3, steps=4, box="configured_strikes")
    F = W.c5_features(2048, 0, N=4, box="configured_strikes")
    assert len(np.unique(F[:, 3])) == 9
    train = [W.c5_instance_from(f, **kw) for f in F]
    y = B.solve_batch(train)
    s = B.Surrogate(members=2, seed=3)
    s.fit(train, y, epochs=4, lr=3e-3)
    s.calibrate(train[:256], y[:256], rel_bound=1e-3, quantile=0.9)
    q = np.array(F[:8])
    q[4:, 3] = q[4:, 3] + 0.5 * (0.04 - 0.02) / 8  # halfway between lattice strikes
    q[4:, 3] = np.minimum(q[4:, 3], 0.0399)
    _, _, in_box = s.predict_features(q)
    assert in_box[:4].all() and not in_box[4:].any(), in_box
    p, fell = s.eval_features(q)
    assert fell[4:].all()
    ref = B.solve_batch([W.c5_instance_from(f, **kw) for f in q[4:]])
    assert np.array_equal(p[4:], ref)
    s.close()
