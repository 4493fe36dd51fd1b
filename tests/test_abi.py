"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every function include/amfrw.h declares, and rejects invalid problem
statements on the host before any CUDA call."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD
from paper_2408_00559_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    BLD.build()
    return B.lib()


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "amfrw.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(amfrw_\w+)\s*\(", hdr)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(B.EXPORTS)


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_status_strings(L):
    for code, name in B.STATUS.items():
        assert L.amfrw_status_string(code).decode() == name
    assert L.amfrw_status_string(99).decode() == "AMFRW_UNKNOWN"


def _expect(inst, status, match=None):
    with pytest.raises(B.AmfrwError) as e:
        B.solve_batch([inst])
    assert e.value.status == status, str(e.value)
    if match:
        assert match in str(e.value)


def test_rejects_non_psd_correlation(L):
    inst = W.small_instance(4, 3)
    inst["phi"] = np.array([-0.9, 0.9, -0.9])
    _expect(inst, 2, "positive semi-definite")


@pytest.mark.parametrize("key,val", [("beta", 1.5), ("n_steps", 0), ("T", -1.0), ("V0", 2.0),
                                     ("sigma", -0.1), ("level", -1), ("nu", 0.0), ("K", float("nan"))])
def test_rejects_bad_scalars(L, key, val):
    inst = W.small_instance(3, 3)
    inst[key] = val
    _expect(inst, 1)


def test_rejects_bad_arrays(L):
    inst = W.small_instance(3, 3)
    inst["F0"] = np.array([0.03, 0.5])  # above Fmax
    _expect(inst, 1)
    inst = W.small_instance(3, 3)
    inst["rho"] = np.array([[1.0, 0.2], [0.3, 1.0]])
    _expect(inst, 1, "symmetric")


def test_rejects_oversized_grid(L):
    inst = W.small_instance(2, 12, full=True)  # 4096 x 4096 Inner nodes
    _expect(inst, 7)


def test_rejects_null_arguments(L):
    assert L.amfrw_solve_batch(None, 1, None, None) == 1
    assert L.amfrw_solve_batch_io(None, None) == 1
    L.amfrw_solve_batch_release()  # nothing kept: a no-op
    assert L.amfrw_batch_run(None, None) == 1
    assert L.amfrw_step(None, 1) == 1
    out = C.c_void_p(1)
    assert L.amfrw_problem_create(None, None, C.byref(out)) == 1
    assert out.value is None


def test_rejects_empty_and_negative_batches(L):
    # an empty problem set is an argument error, reported before any CUDA call
    m = B._Marshal([W.small_instance(3, 3)])
    prices = np.zeros(1)
    out = C.c_void_p(1)
    for n in (0, -1):
        assert L.amfrw_solve_batch(m.arr, n, B._dp(prices), None) == 1
        assert L.amfrw_solve_noalloc(m.arr, n, C.c_void_p(1), None) == 1
        assert L.amfrw_batch_create(m.arr, n, None, C.byref(out)) == 1
        assert out.value is None
        assert "at least one instance" in L.amfrw_last_error().decode()
