"""Oracle: plain serial FP64 CPU reference of the AMFR-W2 / sparse-grid method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The CUDA library in
``paper_2408_00559_gb300`` never imports, links or calls it, and shares no code
with it.  The arithmetic lives in ``amfrw_oracle.c`` (each routine cites the
paper's passage it follows); this module only compiles it with gcc and
marshals arguments through ctypes.

Parity status: every exported routine is pinned by ``tests/test_oracle_*.py``
against something other than itself (closed forms, the paper's printed tables,
dense linear algebra, matrix exponentials, union point counts).
"""
from __future__ import annotations

import ctypes as C
import multiprocessing as mp
import os
import subprocess
import threading

import numpy as np

MAXD = 8
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amfrw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("N", C.c_int32),
        ("payoff", C.c_int32),
        ("n_steps", C.c_int32),
        ("bc", C.c_int32),
        ("alpha", C.c_double * MAXD),
        ("phi", C.c_double * MAXD),
        ("tau", C.c_double * MAXD),
        ("F0", C.c_double * MAXD),
        ("Fmax", C.c_double * MAXD),
        ("rho", C.c_double * (MAXD * MAXD)),
        ("sigma", C.c_double),
        ("beta", C.c_double),
        ("V0", C.c_double),
        ("K", C.c_double),
        ("T", C.c_double),
        ("theta", C.c_double),
        ("nu", C.c_double),
        ("discount", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``amfrw_oracle.c`` into ``liboracle.so`` (gcc, no fast-math)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        pp = C.POINTER(OrcParams)
        L.orc_grid_size.restype = C.c_long
        L.orc_grid_size.argtypes = [C.c_int32, ip]
        L.orc_payoff_grid.argtypes = [pp, ip, dp]
        L.orc_apply_F.argtypes = [pp, ip, dp, dp]
        L.orc_apply_Fi.argtypes = [pp, ip, C.c_int32, dp, dp]
        L.orc_line_solve.argtypes = [pp, ip, C.c_int32, C.c_double, dp, dp]
        L.orc_run.argtypes = [pp, ip, dp, C.c_int32]
        L.orc_run_theta_gs.restype = C.c_int32
        L.orc_run_theta_gs.argtypes = [pp, ip, dp, C.c_int32, C.c_int32]
        L.orc_interp.restype = C.c_double
        L.orc_interp.argtypes = [pp, ip, dp, dp]
        L.orc_solve_grid.restype = C.c_double
        L.orc_solve_grid.argtypes = [pp, ip, dp]
        L.orc_enumerate.restype = C.c_int32
        L.orc_enumerate.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, ip, dp]
        L.orc_price.restype = C.c_double
        L.orc_price.argtypes = [pp, C.c_int32, C.c_int32, C.c_int32, dp]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(inst: dict) -> OrcParams:
    """Fill the oracle's parameter struct from a plain instance dict.

    Keys: N, payoff ('caplet'|'swaption'), n_steps, alpha, phi, tau, F0, Fmax,
    Vmax, rho (n_rates x n_rates), sigma, beta, V0, K, T, theta, nu, discount;
    optional bc ('neumann', the default: Sketch 1; 'dirichlet': eq. bound1_0).
    """
    p = OrcParams()
    N = int(inst["N"])
    nr = N - 1
    p.N = N
    p.payoff = {"caplet": 0, "swaption": 1}[inst["payoff"]]
    p.n_steps = int(inst["n_steps"])
    p.bc = {"neumann": 0, "dirichlet": 1}[inst.get("bc", "neumann")]
    for name in ("alpha", "phi", "tau", "F0"):
        v = np.asarray(inst[name], dtype=np.float64)
        assert v.shape == (nr,), (name, v.shape)
        arr = getattr(p, name)
        for i in range(nr):
            arr[i] = float(v[i])
    fm = np.asarray(inst["Fmax"], dtype=np.float64)
    for i in range(nr):
        p.Fmax[i] = float(fm[i])
    p.Fmax[N - 1] = float(inst["Vmax"])
    rho = np.asarray(inst["rho"], dtype=np.float64).reshape(nr, nr)
    for i in range(nr):
        for k in range(nr):
            p.rho[i * MAXD + k] = float(rho[i, k])
    for name in ("sigma", "beta", "V0", "K", "T", "theta", "nu", "discount"):
        setattr(p, name, float(inst[name]))
    return p


def grid_size(N: int, levels) -> int:
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    return int(lib().orc_grid_size(N, _ip(lv)))


def grid_shape(levels):
    """Node counts per axis, axis 1 first (M_i + 1 each)."""
    return tuple((1 << int(l)) + 1 for l in levels)


def payoff_grid(inst: dict, levels) -> np.ndarray:
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.zeros(grid_size(p.N, lv))
    lib().orc_payoff_grid(C.byref(p), _ip(lv), _dp(Y))
    return Y


def apply_F(inst: dict, levels, Y: np.ndarray) -> np.ndarray:
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros_like(Y)
    lib().orc_apply_F(C.byref(p), _ip(lv), _dp(Y), _dp(out))
    return out


def apply_Fi(inst: dict, levels, axis: int, Y: np.ndarray) -> np.ndarray:
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros_like(Y)
    lib().orc_apply_Fi(C.byref(p), _ip(lv), int(axis), _dp(Y), _dp(out))
    return out


def line_solve(inst: dict, levels, axis: int, nu_dt: float, G: np.ndarray) -> np.ndarray:
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    G = np.ascontiguousarray(G, dtype=np.float64)
    K = np.zeros_like(G)
    lib().orc_line_solve(C.byref(p), _ip(lv), int(axis), float(nu_dt), _dp(G), _dp(K))
    return K


def run(inst: dict, levels, Y0: np.ndarray, n_steps: int | None = None) -> np.ndarray:
    """AMFR-W2 from the full-grid vector Y0 with dt = T / inst['n_steps']."""
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.array(Y0, dtype=np.float64, copy=True)
    lib().orc_run(C.byref(p), _ip(lv), _dp(Y), int(p.n_steps if n_steps is None else n_steps))
    return Y


def run_theta_gs(inst: dict, levels, Y0: np.ndarray, s_iter: int, n_steps: int | None = None) -> np.ndarray:
    """theta-method + Gauss-Seidel W-method (Sec. 4.2) with s_iter iterations
    per step, theta = inst['theta'], dt = T / inst['n_steps'] (small grids)."""
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.array(Y0, dtype=np.float64, copy=True)
    rc = lib().orc_run_theta_gs(C.byref(p), _ip(lv), _dp(Y),
                                int(p.n_steps if n_steps is None else n_steps), int(s_iter))
    if rc != 0:
        raise ValueError("theta-GS oracle: grid above 4096 nodes or s_iter < 1")
    return Y


def interp(inst: dict, levels, Y: np.ndarray, x) -> float:
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    xx = np.zeros(MAXD)
    xx[: len(x)] = x
    return float(lib().orc_interp(C.byref(p), _ip(lv), _dp(Y), _dp(xx)))


def solve_grid(inst: dict, levels, want_Y: bool = False):
    p = make_params(inst)
    lv = np.ascontiguousarray(levels, dtype=np.int32)
    if want_Y:
        Y = np.zeros(grid_size(p.N, lv))
        u = lib().orc_solve_grid(C.byref(p), _ip(lv), _dp(Y))
        return float(u), Y
    return float(lib().orc_solve_grid(C.byref(p), _ip(lv), None))


def enumerate_grids(d: int, n: int, psi: int = 0, full: bool = False):
    """(levels [ng, d] int32, coefs [ng] float64) in the oracle's order."""
    L = lib()
    ng = int(L.orc_enumerate(d, n, psi, int(full), None, None))
    lv = np.zeros((ng, d), dtype=np.int32)
    cf = np.zeros(ng)
    L.orc_enumerate(d, n, psi, int(full), _ip(lv), _dp(cf))
    return lv, cf


def price(inst: dict, n: int, psi: int = 0, full: bool = False, per_grid: bool = False):
    p = make_params(inst)
    L = lib()
    if per_grid:
        ng = int(L.orc_enumerate(p.N, n, psi, int(full), None, None))
        u = np.zeros(ng)
        v = float(L.orc_price(C.byref(p), n, psi, int(full), _dp(u)))
        return v, u
    return float(L.orc_price(C.byref(p), n, psi, int(full), None))


def _grid_value(job):
    inst, levels = job
    return solve_grid(inst, levels)


def price_parallel(inst: dict, n: int, psi: int = 0, full: bool = False, workers: int | None = None) -> float:
    """orc_price with the component grids solved in a spawned process pool
    (largest grids first); the combination sum discount * sum_l c_l u_l then
    runs here in enumeration order, the same sequence of FP64 roundings as
    orc_price.  For the paper-size problems whose serial oracle takes minutes.
    Spawned workers never touch CUDA, so callers may hold a CUDA context."""
    lv, cf = enumerate_grids(int(inst["N"]), n, psi, full)
    sizes = [int(np.prod([(1 << int(x)) + 1 for x in l])) for l in lv]
    order = sorted(range(len(lv)), key=lambda k: -sizes[k])
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or os.cpu_count() or 1) as pool:
        vals = pool.map(_grid_value, [(inst, [int(x) for x in lv[k]]) for k in order], chunksize=1)
    u = [0.0] * len(lv)
    for k, v in zip(order, vals):
        u[k] = v
    s = 0.0
    for k in range(len(lv)):
        s += float(cf[k]) * u[k]
    return float(inst["discount"]) * s
