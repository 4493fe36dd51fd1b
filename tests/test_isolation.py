"""The CUDA path and the CPU oracle stay independent.

The product package (Python binding, CUDA sources and headers under
paper_2408_00559_gb300/ and include/) never imports, includes, loads or names
anything under oracle/, and the oracle never refers to the package, its
kernels or its headers; only the seeded input generators (workloads.py, which
holds no arithmetic of the method) are shared, by the tests.  Without the
compiled library the binding raises instead of falling back to the CPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2408_00559_gb300")


def _files(top, exts):
    for d, _, names in os.walk(top):
        if "__pycache__" in d:
            continue
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def _code(path):
    """Source text without comments and docstrings, so that a sentence that
    mentions the oracle does not count as a use of it."""
    src = open(path, encoding="utf-8").read()
    if path.endswith(".py"):
        src = re.sub(r'"""[\s\S]*?"""', "", src)
        src = re.sub(r"#[^\n]*", "", src)
    else:
        src = re.sub(r"/\*[\s\S]*?\*/", "", src)
        src = re.sub(r"//[^\n]*", "", src)
    return src


def test_product_code_never_uses_the_oracle():
    bad = re.compile(r"\boracle\b|amfrw_oracle|liborc|orc_")
    files = list(_files(PKG, (".py", ".cu", ".cuh", ".h"))) + list(
        _files(os.path.join(ROOT, "include"), (".h",)))
    assert files
    for f in files:
        if os.path.basename(f) == "workloads.py":
            continue  # the shared seeded generators; checked below
        hits = bad.findall(_code(f))
        assert not hits, (os.path.relpath(f, ROOT), hits)


def test_oracle_never_uses_the_product_code():
    bad = re.compile(r"paper_2408_00559_gb300|amfrw\.h|amfrw_internal|libamfrw|csrc")
    files = list(_files(os.path.join(ROOT, "oracle"), (".py", ".c", ".h")))
    assert files
    for f in files:
        hits = bad.findall(_code(f))
        assert not hits, (os.path.relpath(f, ROOT), hits)


def test_shared_generators_hold_no_method_code():
    # workloads.py draws inputs only: it imports neither side
    src = _code(os.path.join(PKG, "workloads.py"))
    assert not re.findall(r"^\s*(?:import|from)\s+(?:oracle|\.|paper_2408_00559_gb300)", src, re.M)
    assert "ctypes" not in src and "CDLL" not in src


def test_binding_fails_loudly_without_the_library(monkeypatch):
    from paper_2408_00559_gb300 import _lib as B
    from paper_2408_00559_gb300 import workloads as W
    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libamfrw.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.solve_batch([W.small_instance(3, 3)])
