"""ctypes binding of libamfrw.so (include/amfrw.h).  Argument marshalling only:
every step of the method runs in the library's CUDA kernels.

The library is loaded from this package directory.  If it is missing the
binding raises; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamfrw.so")

AMFRW_OK = 0
STATUS = {0: "AMFRW_OK", 1: "AMFRW_EINVAL", 2: "AMFRW_ENOTPSD", 3: "AMFRW_ENOMEM",
          4: "AMFRW_ECUDA", 5: "AMFRW_ETIMEOUT", 6: "AMFRW_ENONFINITE", 7: "AMFRW_ETOOBIG"}
PAYOFF = {"caplet": 0, "swaption": 1}
PRECISION = {"fp64": 0, "mixed": 1}
FLAG_GLOBAL_GRIDS = 1
FLAG_DIRICHLET = 2

# every symbol include/amfrw.h declares
EXPORTS = [
    "amfrw_problem_create", "amfrw_step", "amfrw_combine", "amfrw_problem_num_grids",
    "amfrw_problem_grid_info", "amfrw_problem_grid_values", "amfrw_problem_read_grid",
    "amfrw_problem_destroy", "amfrw_solve_batch", "amfrw_batch_create", "amfrw_batch_run",
    "amfrw_batch_launches", "amfrw_batch_destroy", "amfrw_status_string", "amfrw_last_error",
    "amfrw_batch_enable_timing", "amfrw_batch_kernel_times", "amfrw_batch_io_bytes",
    "amfrw_solve_noalloc", "amfrw_batch_autotune", "amfrw_batch_classes", "amfrw_tc_gemm_bf16",
    "amfrw_surrogate_create", "amfrw_surrogate_fit", "amfrw_surrogate_calibrate",
    "amfrw_surrogate_predict", "amfrw_surrogate_predict_features", "amfrw_surrogate_eval",
    "amfrw_surrogate_eval_features",
    "amfrw_surrogate_save",
    "amfrw_surrogate_load", "amfrw_surrogate_params", "amfrw_surrogate_grad",
    "amfrw_surrogate_destroy", "amfrw_surrogate_last_error", "amfrw_peak_probe",
    "amfrw_batch_set_kappa_max", "amfrw_batch_promoted", "amfrw_solve_batch_io",
    "amfrw_solve_batch_release",
]
SURROGATE_PARAMS = 136193


class AmfrwError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")


class Params(C.Structure):
    _fields_ = [
        ("n_rates", C.c_int32), ("payoff", C.c_int32), ("n_steps", C.c_int32),
        ("level", C.c_int32), ("psi", C.c_int32), ("full_grid", C.c_int32),
        ("precision", C.c_int32), ("flags", C.c_int32),
        ("alpha", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double)),
        ("rho", C.POINTER(C.c_double)), ("tau", C.POINTER(C.c_double)),
        ("F0", C.POINTER(C.c_double)), ("Fmax", C.POINTER(C.c_double)),
        ("sigma", C.c_double), ("beta", C.c_double), ("V0", C.c_double), ("Vmax", C.c_double),
        ("K", C.c_double), ("T", C.c_double), ("discount", C.c_double), ("theta", C.c_double),
        ("nu_amf", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing; build it with "
                "`python -m paper_2408_00559_gb300.build` (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        pp = C.POINTER(Params)
        L.amfrw_problem_create.argtypes = [pp, vp, C.POINTER(vp)]
        L.amfrw_step.argtypes = [vp, C.c_int32]
        L.amfrw_combine.argtypes = [vp, C.POINTER(C.c_double)]
        L.amfrw_problem_num_grids.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.amfrw_problem_grid_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.amfrw_problem_grid_values.argtypes = [vp, C.POINTER(C.c_double)]
        L.amfrw_problem_read_grid.argtypes = [vp, C.c_int32, C.POINTER(C.c_double)]
        L.amfrw_problem_destroy.argtypes = [vp]
        L.amfrw_problem_destroy.restype = None
        L.amfrw_solve_batch.argtypes = [pp, C.c_int32, C.POINTER(C.c_double), vp]
        L.amfrw_solve_batch_io.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.amfrw_solve_batch_release.argtypes = []
        L.amfrw_solve_batch_release.restype = None
        L.amfrw_batch_create.argtypes = [pp, C.c_int32, vp, C.POINTER(vp)]
        L.amfrw_batch_run.argtypes = [vp, vp]
        L.amfrw_batch_launches.argtypes = [vp, C.POINTER(C.c_int32)]
        L.amfrw_batch_destroy.argtypes = [vp]
        L.amfrw_batch_destroy.restype = None
        L.amfrw_batch_enable_timing.argtypes = [vp, C.c_int32]
        L.amfrw_batch_kernel_times.argtypes = [vp, C.POINTER(C.c_float), C.POINTER(C.c_double),
                                               C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)]
        L.amfrw_batch_io_bytes.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.amfrw_solve_noalloc.argtypes = [pp, C.c_int32, vp, vp]
        L.amfrw_peak_probe.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double), vp]
        L.amfrw_batch_set_kappa_max.argtypes = [vp, C.c_double]
        L.amfrw_batch_promoted.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        L.amfrw_batch_autotune.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
        L.amfrw_batch_classes.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        i32 = C.c_int32
        L.amfrw_tc_gemm_bf16.argtypes = [vp, i32, vp, i32, vp, i32, i32, i32, i32, vp]
        i64, u8p, fp = C.c_int64, C.POINTER(C.c_uint8), C.POINTER(C.c_float)
        dpp = C.POINTER(C.c_double)
        L.amfrw_surrogate_create.argtypes = [i32, C.c_uint64, vp, C.POINTER(vp)]
        L.amfrw_surrogate_fit.argtypes = [vp, pp, dpp, i64, i32, C.c_float, fp]
        L.amfrw_surrogate_calibrate.argtypes = [vp, pp, dpp, i64, C.c_double, C.c_double, dpp]
        L.amfrw_surrogate_predict.argtypes = [vp, pp, i64, dpp, dpp, u8p]
        L.amfrw_surrogate_eval.argtypes = [vp, pp, i64, dpp, u8p, vp]
        L.amfrw_surrogate_eval_features.argtypes = [vp, dpp, i64, dpp, u8p, vp]
        L.amfrw_surrogate_predict_features.argtypes = [vp, dpp, i64, dpp, dpp, u8p]
        L.amfrw_surrogate_save.argtypes = [vp, C.c_char_p]
        L.amfrw_surrogate_load.argtypes = [C.c_char_p, vp, C.POINTER(vp)]
        L.amfrw_surrogate_params.argtypes = [vp, i32, fp, fp]
        L.amfrw_surrogate_grad.argtypes = [vp, i32, fp, fp, i32, fp, fp]
        L.amfrw_surrogate_destroy.argtypes = [vp]
        L.amfrw_surrogate_destroy.restype = None
        L.amfrw_surrogate_last_error.restype = C.c_char_p
        L.amfrw_surrogate_last_error.argtypes = []
        L.amfrw_status_string.restype = C.c_char_p
        L.amfrw_status_string.argtypes = [C.c_int]
        L.amfrw_last_error.restype = C.c_char_p
        L.amfrw_last_error.argtypes = []
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != AMFRW_OK:
        raise AmfrwError(rc, where, lib().amfrw_last_error().decode())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Marshal:
    """amfrw_params records for a list of instance dicts; keeps the arrays alive."""

    def __init__(self, insts: list[dict]):
        self.keep = []
        self.arr = (Params * len(insts))()
        for k, inst in enumerate(insts):
            self._fill(self.arr[k], inst)

    def _vec(self, x) -> np.ndarray:
        a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
        self.keep.append(a)
        return a

    def _fill(self, p: Params, inst: dict):
        N = int(inst["N"])
        p.n_rates = N - 1
        p.payoff = PAYOFF[inst["payoff"]]
        p.n_steps = int(inst["n_steps"])
        p.level = int(inst["level"])
        p.psi = int(inst.get("psi", 0))
        p.full_grid = int(bool(inst.get("full", False)))
        p.precision = PRECISION[inst.get("precision", "fp64")]
        p.flags = ((FLAG_GLOBAL_GRIDS if inst.get("global_grids", False) else 0) |
                   (FLAG_DIRICHLET if inst.get("bc", "neumann") == "dirichlet" else 0))
        for name in ("alpha", "phi", "tau", "F0", "Fmax"):
            setattr(p, name, _dp(self._vec(inst[name])))
        p.rho = _dp(self._vec(inst["rho"]))
        p.sigma = float(inst["sigma"])
        p.beta = float(inst["beta"])
        p.V0 = float(inst["V0"])
        p.Vmax = float(inst["Vmax"])
        p.K = float(inst["K"])
        p.T = float(inst["T"])
        p.discount = float(inst.get("discount", 1.0))
        p.theta = float(inst["theta"])
        p.nu_amf = float(inst["nu"])


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return int(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class Problem:
    """amfrw_problem: one instance, stepped in time, state kept on the device."""

    def __init__(self, inst: dict, stream=None):
        self._m = _Marshal([inst])
        self.h = C.c_void_p()
        _check(lib().amfrw_problem_create(self._m.arr, _stream_ptr(stream), C.byref(self.h)),
               "amfrw_problem_create")
        ng, dim = C.c_int32(), C.c_int32()
        _check(lib().amfrw_problem_num_grids(self.h, C.byref(ng), C.byref(dim)),
               "amfrw_problem_num_grids")
        self.n_grids, self.dim = ng.value, dim.value

    def step(self, n_steps: int):
        _check(lib().amfrw_step(self.h, int(n_steps)), "amfrw_step")

    def combine(self) -> float:
        v = C.c_double()
        _check(lib().amfrw_combine(self.h, C.byref(v)), "amfrw_combine")
        return v.value

    def grid_info(self):
        lv = np.zeros((self.n_grids, self.dim), dtype=np.int32)
        cf = np.zeros(self.n_grids)
        _check(lib().amfrw_problem_grid_info(self.h, lv.ctypes.data_as(C.POINTER(C.c_int32)), _dp(cf)),
               "amfrw_problem_grid_info")
        return lv, cf

    def grid_values(self) -> np.ndarray:
        u = np.zeros(self.n_grids)
        _check(lib().amfrw_problem_grid_values(self.h, _dp(u)), "amfrw_problem_grid_values")
        return u

    def read_grid(self, g: int, levels) -> np.ndarray:
        L = int(np.prod([1 << int(x) for x in levels]))
        Y = np.zeros(L)
        _check(lib().amfrw_problem_read_grid(self.h, int(g), _dp(Y)), "amfrw_problem_read_grid")
        return Y

    def close(self):
        if self.h:
            lib().amfrw_problem_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(insts: list[dict], stream=None) -> np.ndarray:
    """amfrw_solve_batch: host params in, host prices out."""
    m = _Marshal(insts)
    out = np.zeros(len(insts))
    _check(lib().amfrw_solve_batch(m.arr, len(insts), _dp(out), _stream_ptr(stream)),
           "amfrw_solve_batch")
    return out


def solve_batch_io() -> tuple[int, int]:
    """amfrw_solve_batch_io: (host->device, device->host) bytes of this thread's last solve_batch."""
    h, d = C.c_int64(), C.c_int64()
    _check(lib().amfrw_solve_batch_io(C.byref(h), C.byref(d)), "amfrw_solve_batch_io")
    return h.value, d.value


def solve_batch_release() -> None:
    """amfrw_solve_batch_release: free the plan solve_batch keeps for this thread."""
    lib().amfrw_solve_batch_release()


class Batch:
    """amfrw_batch: inputs uploaded once, run() prices into a device array."""

    def __init__(self, insts: list[dict], stream=None):
        self._m = _Marshal(insts)
        self.n = len(insts)
        self.h = C.c_void_p()
        _check(lib().amfrw_batch_create(self._m.arr, self.n, _stream_ptr(stream), C.byref(self.h)),
               "amfrw_batch_create")

    def run(self, d_prices_ptr: int):
        _check(lib().amfrw_batch_run(self.h, C.c_void_p(int(d_prices_ptr))), "amfrw_batch_run")

    def launches(self) -> int:
        n = C.c_int32()
        _check(lib().amfrw_batch_launches(self.h, C.byref(n)), "amfrw_batch_launches")
        return n.value

    def enable_timing(self, on: bool = True):
        _check(lib().amfrw_batch_enable_timing(self.h, int(bool(on))), "amfrw_batch_enable_timing")

    def kernel_times(self):
        """[(N, device ms, Inner-node-steps)] of each solver launch of the last run."""
        cap = 64
        ms = (C.c_float * cap)()
        ns = (C.c_double * cap)()
        dims = (C.c_int32 * cap)()
        n = C.c_int32()
        _check(lib().amfrw_batch_kernel_times(self.h, ms, ns, dims, cap, C.byref(n)),
               "amfrw_batch_kernel_times")
        return [(dims[i], ms[i], ns[i]) for i in range(n.value)]

    def set_kappa_max(self, kappa_max: float):
        """Condition bound above which mixed instances are re-solved in FP64
        inside the batch's graph (<= 0: off)."""
        _check(lib().amfrw_batch_set_kappa_max(self.h, float(kappa_max)), "amfrw_batch_set_kappa_max")

    def promoted(self):
        """(instances re-solved in FP64 by the last run, kappa per instance)."""
        n = C.c_int32()
        kappa = np.zeros(self.n)
        _check(lib().amfrw_batch_promoted(self.h, C.byref(n), _dp(kappa)), "amfrw_batch_promoted")
        return n.value, kappa

    def autotune(self, trials: int = 2) -> bool:
        """Pick the faster launch strategy and grid-state placement on this
        device; True = one persistent multi-class launch for the warp-solved
        grids."""
        m = C.c_int32()
        _check(lib().amfrw_batch_autotune(self.h, int(trials), C.byref(m)), "amfrw_batch_autotune")
        return bool(m.value)

    def classes(self):
        """Launch classes by kind: (warp groups, CTA groups, global-memory groups)."""
        w, c, g = C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().amfrw_batch_classes(self.h, C.byref(w), C.byref(c), C.byref(g)), "amfrw_batch_classes")
        return w.value, c.value, g.value

    def io_bytes(self):
        h2d, d2h = C.c_int64(), C.c_int64()
        _check(lib().amfrw_batch_io_bytes(self.h, C.byref(h2d), C.byref(d2h)), "amfrw_batch_io_bytes")
        return h2d.value, d2h.value

    def close(self):
        if self.h:
            lib().amfrw_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_noalloc(insts: list[dict], d_prices_ptr: int, stream=None):
    """amfrw_solve_noalloc: prices into the device array at d_prices_ptr
    without any device allocation by the library (its working memory is a
    fixed array inside the library, shared by all calls; see include/amfrw.h
    for the size limit and why overlapping calls must be serialised)."""
    m = _Marshal(insts)
    _check(lib().amfrw_solve_noalloc(m.arr, len(insts), C.c_void_p(int(d_prices_ptr)),
                                     _stream_ptr(stream)), "amfrw_solve_noalloc")


def peak_probe(precision: str = "fp64", iters: int = 4096, stream=None) -> float:
    """amfrw_peak_probe: measured FMA throughput of the current device in
    TFLOP/s for precision 'fp64' or 'fp32'."""
    out = C.c_double(0.0)
    code = {"fp64": 0, "fp32": 2}[precision]
    _check(lib().amfrw_peak_probe(code, int(iters), C.byref(out), _stream_ptr(stream)), "amfrw_peak_probe")
    return float(out.value)


def tc_gemm_bf16(A, B, C, stream=None):
    """C = A @ B.T on the tensor cores; A [M,K], B [N,K] BF16, C [M,N] FP32
    CUDA tensors (row-major, contiguous)."""
    M, K = A.shape
    N = B.shape[0]
    _check(lib().amfrw_tc_gemm_bf16(C_void(A.data_ptr()), A.stride(0), C_void(B.data_ptr()), B.stride(0),
                                    C_void(C.data_ptr()), C.stride(0), M, N, K, _stream_ptr(stream)),
           "amfrw_tc_gemm_bf16")


def C_void(p):
    return C.c_void_p(int(p))


def _scheck(rc: int, where: str):
    if rc != AMFRW_OK:
        raise AmfrwError(rc, where, lib().amfrw_surrogate_last_error().decode())


def _fp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class Surrogate:
    """amfrw_surrogate: an ensemble of MLPs trained on solver prices, with the
    batched solver as fallback (see include/amfrw.h)."""

    def __init__(self, members: int = 4, seed: int = 0, stream=None, _handle=None):
        self.stream = stream
        if _handle is not None:
            self.h = _handle
            return
        self.h = C.c_void_p()
        _scheck(lib().amfrw_surrogate_create(int(members), int(seed), _stream_ptr(stream), C.byref(self.h)),
                "amfrw_surrogate_create")

    def fit(self, insts, prices, epochs: int = 40, lr: float = 2e-3) -> float:
        m = _Marshal(insts)
        pr = np.ascontiguousarray(prices, dtype=np.float64)
        loss = C.c_float()
        _scheck(lib().amfrw_surrogate_fit(self.h, m.arr, _dp(pr), len(insts), int(epochs), float(lr),
                                          C.byref(loss)), "amfrw_surrogate_fit")
        return loss.value

    def calibrate(self, insts, prices, rel_bound: float = 1e-3, quantile: float = 0.99) -> float:
        m = _Marshal(insts)
        pr = np.ascontiguousarray(prices, dtype=np.float64)
        c = C.c_double()
        _scheck(lib().amfrw_surrogate_calibrate(self.h, m.arr, _dp(pr), len(insts), float(rel_bound),
                                                float(quantile), C.byref(c)), "amfrw_surrogate_calibrate")
        return c.value

    def predict(self, insts):
        m = _Marshal(insts)
        n = len(insts)
        mean, spread = np.zeros(n), np.zeros(n)
        ok = np.zeros(n, dtype=np.uint8)
        _scheck(lib().amfrw_surrogate_predict(self.h, m.arr, n, _dp(mean), _dp(spread),
                                              ok.ctypes.data_as(C.POINTER(C.c_uint8))),
                "amfrw_surrogate_predict")
        return mean, spread, ok.astype(bool)

    def predict_features(self, features):
        f = np.ascontiguousarray(features, dtype=np.float64)
        n = f.shape[0]
        mean, spread = np.zeros(n), np.zeros(n)
        ok = np.zeros(n, dtype=np.uint8)
        _scheck(lib().amfrw_surrogate_predict_features(self.h, _dp(f), n, _dp(mean), _dp(spread),
                                                       ok.ctypes.data_as(C.POINTER(C.c_uint8))),
                "amfrw_surrogate_predict_features")
        return mean, spread, ok.astype(bool)

    def eval(self, insts, marshalled=None):
        m = marshalled if marshalled is not None else _Marshal(insts)
        n = len(insts) if insts is not None else len(m.arr)
        prices = np.zeros(n)
        fell = np.zeros(n, dtype=np.uint8)
        _scheck(lib().amfrw_surrogate_eval(self.h, m.arr, n, _dp(prices),
                                           fell.ctypes.data_as(C.POINTER(C.c_uint8)),
                                           _stream_ptr(self.stream)), "amfrw_surrogate_eval")
        return prices, fell.astype(bool)

    def eval_features(self, features):
        """Queries given as raw features [n x 8] of the family's instances."""
        f = np.ascontiguousarray(features, dtype=np.float64)
        n = f.shape[0]
        prices = np.zeros(n)
        fell = np.zeros(n, dtype=np.uint8)
        _scheck(lib().amfrw_surrogate_eval_features(self.h, _dp(f), n, _dp(prices),
                                                    fell.ctypes.data_as(C.POINTER(C.c_uint8)),
                                                    _stream_ptr(self.stream)), "amfrw_surrogate_eval_features")
        return prices, fell.astype(bool)

    def save(self, path: str):
        _scheck(lib().amfrw_surrogate_save(self.h, str(path).encode()), "amfrw_surrogate_save")

    @staticmethod
    def load(path: str, stream=None) -> "Surrogate":
        h = C.c_void_p()
        _scheck(lib().amfrw_surrogate_load(str(path).encode(), _stream_ptr(stream), C.byref(h)),
                "amfrw_surrogate_load")
        return Surrogate(stream=stream, _handle=h)

    def params(self, member: int = 0, new=None) -> np.ndarray:
        out = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
        src = None
        if new is not None:
            src = np.ascontiguousarray(new, dtype=np.float32)
            assert src.size == SURROGATE_PARAMS
        _scheck(lib().amfrw_surrogate_params(self.h, int(member), _fp(out),
                                             _fp(src) if src is not None else None),
                "amfrw_surrogate_params")
        return out

    def grad(self, member: int, x_norm, targets):
        x = np.ascontiguousarray(x_norm, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        g = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
        loss = C.c_float()
        _scheck(lib().amfrw_surrogate_grad(self.h, int(member), _fp(x), _fp(t), x.shape[0], _fp(g),
                                           C.byref(loss)), "amfrw_surrogate_grad")
        return g, loss.value

    def close(self):
        if self.h:
            lib().amfrw_surrogate_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surrogate_layout():
    """Offsets of the FP32 parameter vector of one member."""
    W, P = 256, 16
    o = {}
    off = 0
    for name, size in (("W1", W * P), ("b1", W), ("W2", W * W), ("b2", W), ("W3", W * W), ("b3", W),
                       ("w4", W), ("b4", 1)):
        o[name] = (off, size)
        off += size
    assert off == SURROGATE_PARAMS
    return o
