"""The seeded input recipe that both the CUDA path and the oracle draw from
(paper_2408_00559_gb300/workloads.py): every configuration has the shapes,
ranges and structure its description states, the draws are reproducible from
the instance index alone, and every joint correlation matrix of
(F_1..F_{N-1}, V) is positive semi-definite (Sec. 2 needs a valid correlation
for the SABR-LMM dynamics)."""
import numpy as np
import pytest

from paper_2408_00559_gb300 import workloads as W

THETA = (3.0 + np.sqrt(3.0)) / 6.0


def joint_min_eig(inst):
    n = inst["N"] - 1
    C = np.eye(n + 1)
    C[:n, :n] = inst["rho"]
    C[:n, n] = inst["phi"]
    C[n, :n] = inst["phi"]
    return np.linalg.eigvalsh(C).min()


def check_rates_family(inst, N):
    nr = N - 1
    assert inst["N"] == N and inst["payoff"] == "swaption"
    for key in ("alpha", "phi", "tau", "F0", "Fmax"):
        assert np.shape(inst[key]) == (nr,), key
    assert np.all((inst["alpha"] >= 0.1) & (inst["alpha"] <= 0.4))
    assert 0.1 <= inst["sigma"] <= 0.5
    assert np.all((inst["phi"] >= -0.5) & (inst["phi"] <= 0.0))
    i = np.arange(nr)
    assert np.allclose(inst["rho"], np.exp(-0.1 * np.abs(i[:, None] - i[None, :])), rtol=0, atol=0)
    assert np.all(inst["tau"] == 0.5) and np.all(inst["F0"] == 0.03) and np.all(inst["Fmax"] == 0.2)
    assert inst["K"] == 0.03 and inst["beta"] == 0.5 and inst["V0"] == 1.0 and inst["Vmax"] == 1.0
    assert inst["T"] == 2.0 and inst["n_steps"] == 40 and inst["discount"] == 1.0
    assert inst["theta"] == pytest.approx(THETA, abs=0) and inst["nu"] == pytest.approx(0.5 * N * THETA)
    assert joint_min_eig(inst) >= -1e-12


def test_c1_is_the_65x65_full_grid_caplet():
    c = W.c1_instance()
    assert c["N"] == 2 and c["full"] and c["level"] == 6 and c["precision"] == "fp64"
    assert c["payoff"] == "caplet" and c["n_steps"] == 20 and c["K"] == c["F0"][0] == 0.03
    assert (1 << c["level"]) + 1 == 65


def test_c2_and_c3_shapes():
    for idx in range(16):
        c2 = W.c2_instance(idx)
        check_rates_family(c2, 4)
        assert c2["level"] == 5 and c2["psi"] == 0 and not c2["full"] and c2["precision"] == "fp64"
        c3 = W.c3_instance(idx)
        check_rates_family(c3, 6)
        assert c3["level"] == 6 and c3["psi"] == 1 and c3["precision"] == "mixed"


def test_c4_batch_is_uneven_over_every_dimension_and_level():
    b = W.batch("c4", 256)
    assert len(b) == 256
    seen = set()
    for inst in b:
        check_rates_family(inst, inst["N"])
        assert inst["N"] in (4, 6, 8) and inst["level"] in (4, 5, 6)
        assert inst["psi"] == 0 and not inst["full"] and inst["precision"] == "mixed"
        seen.add((inst["N"], inst["level"]))
    assert seen == {(N, n) for N in (4, 6, 8) for n in (4, 5, 6)}


def test_draws_depend_on_the_instance_index_only():
    a = W.batch("c4", 8, start=100)
    b = [W.c4_instance(100 + i) for i in range(8)]
    for x, y in zip(a, b):
        for key in ("alpha", "phi", "sigma", "N", "level"):
            assert np.array_equal(np.asarray(x[key]), np.asarray(y[key])), key
    # neighbouring indices draw different parameters
    assert not np.array_equal(W.c2_instance(0)["alpha"], W.c2_instance(1)["alpha"])
    # the precision switch changes nothing else
    m, f = W.c4_instance(3), W.c4_instance(3, precision="fp64")
    assert f["precision"] == "fp64" and np.array_equal(m["alpha"], f["alpha"]) and m["N"] == f["N"]


@pytest.mark.parametrize("box", ["configured", "configured_strikes", "centred"])
def test_surrogate_features_lie_in_their_box(box):
    B = W.C5_BOXES[box]
    F = W.c5_features(2048, 7, box=box)
    for c, key in enumerate(("alpha", "sigma", "beta", "K", "T", "lam")):
        lo, hi = B[key]
        assert np.all((F[:, c] >= lo) & (F[:, c] <= hi)), key
    assert np.all((F[:, 6:8] >= B["phi"][0]) & (F[:, 6:8] <= B["phi"][1]))
    if box == "configured_strikes":
        lattice = np.linspace(*B["K"], B["K_lattice"])
        assert np.all(np.min(np.abs(F[:, 3, None] - lattice[None, :]), axis=1) <= 1e-15)
        assert len(np.unique(np.round(F[:, 3], 12))) == B["K_lattice"]
    for f in F[:64]:
        inst = W.c5_instance_from(f, box=box)
        nr = inst["N"] - 1
        assert np.all(inst["alpha"] == f[0]) and inst["K"] == f[3] and inst["T"] == f[4]
        assert inst["phi"][0] == f[6] and inst["phi"][nr - 1] == pytest.approx(f[7], abs=1e-15)
        assert np.all(inst["Fmax"] == B["Fmax"]) and inst["Vmax"] == B["Vmax"]
        assert joint_min_eig(inst) >= -1e-12
