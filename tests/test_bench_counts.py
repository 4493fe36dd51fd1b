"""The operation counts behind bench.py's roofline rest on its own grid
enumeration; here it is checked against the oracle's (eqs.
standardCombTechnique / modifiedCombTechnique, whose point counts the oracle
pins to the paper's tables), and the counts against properties they must
have: the mixed split adds up to the FP64 count it partitions, FP64
instances count everything as FP64, and work grows with the steps."""
import os
import sys

import numpy as np
import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2408_00559_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    O.build()


@pytest.mark.parametrize("d,n,psi", [(2, 6, 0), (4, 5, 0), (6, 6, 1), (8, 4, 0), (8, 6, 0), (3, 9, 0), (5, 3, 2)])
def test_bench_enumerates_the_oracles_grids(d, n, psi):
    lv, _ = O.enumerate_grids(d, n, psi)
    mine = sorted(tuple(x) for x in bench.enumerate_levels(d, n, psi))
    theirs = sorted(tuple(int(v) for v in row) for row in lv)
    assert mine == theirs


def test_batched_workload_node_steps():
    """2.1e8 node-steps of the N=8 grids of the 256-instance batch: the
    denominator of the instructions-per-node-step figure of the profile."""
    b = W.batch("c4", 256)
    ns = 0
    for inst in b:
        if inst["N"] != 8:
            continue
        for lv in bench.enumerate_levels(8, inst["level"], 0):
            ns += (1 << int(sum(lv))) * inst["n_steps"]
    assert ns == pytest.approx(2.11e8, rel=0.01)


def test_mixed_split_partitions_the_work():
    for lv in ([1, 0, 2, 1], [0, 0, 0], [2, 2], [1, 1, 1, 1, 1, 1, 0, 0]):
        total = bench.node_flops(lv, 40)
        f32, f64 = bench.mixed_ops(lv, 40)
        L = 1 << sum(lv)
        N = len(lv)
        # FP32 takes everything but the two updates; FP64 the accumulation,
        # F of the payoff and the interpolation
        assert f32 == pytest.approx(total - 6.0 * L * 40)
        assert f64 == pytest.approx(4.0 * L * 40 + bench.payoff_F_flops(lv) + (1 << N) * (3 * N + 2))
        assert bench.node_flops(lv, 80) == pytest.approx(2 * total)
    insts = W.batch("c4", 6)
    f32, f64 = bench.batch_ops([dict(x, precision="fp64") for x in insts])
    assert f32 == 0.0 and f64 > 0
    m32, m64 = bench.batch_ops(insts)
    assert m32 > 0 and 0 < m64 < f64
