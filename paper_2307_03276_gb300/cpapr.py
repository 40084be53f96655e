"""Thin ctypes binding of libcpapr.so (include/cpapr.h).

Argument marshalling only: every step of CP-APR MU runs in the CUDA library.
The functions carry the C names; `Tensor` is a small convenience wrapper
around a context.  Arrays may be numpy arrays (host) or torch tensors (host,
pinned host or CUDA); outputs are numpy arrays unless a torch tensor is
passed as `out`.  There is no CPU fallback: if the library cannot be loaded
every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcpapr.so")
MAX_MODES = 8

CPAPR_FP64, CPAPR_FP32 = 0, 1
CPAPR_REDUCE_AUTO, CPAPR_REDUCE_ATOMIC, CPAPR_REDUCE_SEGMENTED = 0, 1, 2
CPAPR_PI_AUTO, CPAPR_PI_FUSED, CPAPR_PI_MATERIALISED = 0, 1, 2
CPAPR_DOT_AUTO, CPAPR_DOT_FP64, CPAPR_DOT_FP32_PIPE = 0, 1, 2
K_PHI, K_PI, K_UPDATE, K_NORM, K_SB, K_LL, K_MTTKRP = range(7)

STATUS = {0: "CPAPR_OK", 1: "CPAPR_E_ARG", 2: "CPAPR_E_RANGE", 3: "CPAPR_E_VALUE", 4: "CPAPR_E_NOMEM",
          5: "CPAPR_E_CUDA", 6: "CPAPR_E_TIMEOUT", 7: "CPAPR_E_STATE"}
EXPORTS = ["cpapr_default_options", "cpapr_create", "cpapr_destroy", "cpapr_set_model", "cpapr_init_random",
           "cpapr_get_model", "cpapr_phi", "cpapr_mttkrp", "cpapr_loglik", "cpapr_mu_solve", "cpapr_batch_mu_solve",
           "cpapr_get_info", "cpapr_kernel_stats", "cpapr_last_error", "cpapr_version"]


class CpaprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("reduction", ctypes.c_int32), ("eps", ctypes.c_double),
                ("kappa", ctypes.c_double), ("kappa_tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("tile_nnz", ctypes.c_int32), ("rank_lanes", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("autotune", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("pi_mode", ctypes.c_int32), ("l2_persist", ctypes.c_int32), ("fp64_dot", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p)]


class Result(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("total_inner", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("loglik", ctypes.c_double), ("kkt_viol", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {"outer_iters": self.outer_iters, "total_inner": self.total_inner, "converged": bool(self.converged),
                "loglik": self.loglik, "kkt_viol": self.kkt_viol}


class Info(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int32), ("rank", ctypes.c_int32), ("rank_padded", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("nnz", ctypes.c_int64), ("dims", ctypes.c_int64 * MAX_MODES),
                ("tile_nnz", ctypes.c_int32 * MAX_MODES), ("rank_lanes", ctypes.c_int32 * MAX_MODES),
                ("reduction", ctypes.c_int32 * MAX_MODES), ("ntiles", ctypes.c_int32 * MAX_MODES),
                ("nsplit", ctypes.c_int32 * MAX_MODES), ("pi_mode", ctypes.c_int32 * MAX_MODES),
                ("device_bytes", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("l2_window_bytes", ctypes.c_int64)]


_lib = None


def load() -> ctypes.CDLL:
    """Loads libcpapr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: build it with paper_2307_03276_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.cpapr_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.cpapr_default_options.restype = None
    lib.cpapr_create.argtypes = [i32, P, i64, P, P, i32, ctypes.POINTER(Options), ctypes.POINTER(P)]
    lib.cpapr_destroy.argtypes = [P]
    lib.cpapr_destroy.restype = None
    lib.cpapr_set_model.argtypes = [P, P, P]
    lib.cpapr_init_random.argtypes = [P, ctypes.c_uint64]
    lib.cpapr_get_model.argtypes = [P, P, P]
    lib.cpapr_phi.argtypes = [P, i32, P, P]
    lib.cpapr_phi_noalloc.argtypes = [P, i32, P, P]
    lib.cpapr_get_state.argtypes = [P, P, P, P, ctypes.POINTER(i64)]
    lib.cpapr_set_state.argtypes = [P, P, P, P, i64]
    lib.cpapr_mttkrp.argtypes = [P, i32, P]
    lib.cpapr_loglik.argtypes = [P, P]
    lib.cpapr_mu_solve.argtypes = [P, f64, i32, i32, ctypes.POINTER(Result), P, P, P]
    lib.cpapr_batch_mu_solve.argtypes = [P, i32, f64, i32, i32, P]
    lib.cpapr_get_info.argtypes = [P, ctypes.POINTER(Info)]
    lib.cpapr_kernel_stats.argtypes = [P, i32, ctypes.POINTER(i64), ctypes.POINTER(f64), i32]
    lib.cpapr_last_error.argtypes = [P]
    lib.cpapr_last_error.restype = ctypes.c_char_p
    lib.cpapr_version.argtypes = []
    lib.cpapr_version.restype = ctypes.c_char_p
    for name in ("cpapr_create", "cpapr_set_model", "cpapr_init_random", "cpapr_get_model", "cpapr_phi",
                 "cpapr_phi_noalloc", "cpapr_get_state", "cpapr_set_state",
                 "cpapr_mttkrp", "cpapr_loglik", "cpapr_mu_solve", "cpapr_batch_mu_solve", "cpapr_get_info",
                 "cpapr_kernel_stats"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != 0:
        msg = load().cpapr_last_error(ctx).decode()
        raise CpaprError(st, msg)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _as_f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64:
            raise TypeError("expected float64")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64)


def _as_i64(a):
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.int64:
            raise TypeError("expected int64")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.int64)


def cpapr_default_options(**overrides) -> Options:
    o = Options()
    load().cpapr_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(getattr(v, "cuda_stream", v))
        if k == "tune_cache" and v is not None and not isinstance(v, bytes):
            v = os.fsencode(v)
        setattr(o, k, v)
    return o


def cpapr_create(dims, idx, vals, rank: int, opt: Options | None = None):
    """Returns an opaque context handle (int).  idx: [N, nnz] int64 or N arrays."""
    lib = load()
    N = len(dims)
    d = np.ascontiguousarray(dims, dtype=np.int64)
    rows = [_as_i64(idx[m]) for m in range(N)]
    v = _as_f64(vals)
    nnz = int(v.shape[0])
    arr = (ctypes.c_void_p * N)(*[_ptr(r) for r in rows])
    h = ctypes.c_void_p()
    st = lib.cpapr_create(N, d.ctypes.data, nnz, arr, _ptr(v), int(rank), ctypes.byref(opt) if opt else None,
                          ctypes.byref(h))
    _check(st, None)
    return h.value


def cpapr_destroy(ctx) -> None:
    if ctx:
        load().cpapr_destroy(ctx)


def cpapr_set_model(ctx, lam, factors) -> None:
    lam = _as_f64(lam)
    fs = [_as_f64(A) for A in factors]
    arr = (ctypes.c_void_p * len(fs))(*[_ptr(A) for A in fs])
    _check(load().cpapr_set_model(ctx, _ptr(lam), arr), ctx)


def cpapr_init_random(ctx, seed: int) -> None:
    _check(load().cpapr_init_random(ctx, ctypes.c_uint64(seed)), ctx)


def cpapr_get_info(ctx) -> Info:
    info = Info()
    _check(load().cpapr_get_info(ctx, ctypes.byref(info)), ctx)
    return info


def cpapr_get_model(ctx):
    info = cpapr_get_info(ctx)
    R = info.rank
    lam = np.zeros(R)
    fs = [np.zeros((info.dims[m], R)) for m in range(info.nmodes)]
    arr = (ctypes.c_void_p * len(fs))(*[A.ctypes.data for A in fs])
    _check(load().cpapr_get_model(ctx, lam.ctypes.data, arr), ctx)
    return lam, fs


def cpapr_get_state(ctx) -> dict:
    """Checkpoint: lambda, factors, each mode's last Phi and the outer-iteration count."""
    info = cpapr_get_info(ctx)
    R = info.rank
    lam = np.zeros(R)
    fs = [np.zeros((info.dims[m], R)) for m in range(info.nmodes)]
    ph = [np.zeros((info.dims[m], R)) for m in range(info.nmodes)]
    arr_f = (ctypes.c_void_p * len(fs))(*[A.ctypes.data for A in fs])
    arr_p = (ctypes.c_void_p * len(ph))(*[A.ctypes.data for A in ph])
    k = ctypes.c_int64()
    _check(load().cpapr_get_state(ctx, lam.ctypes.data, arr_f, arr_p, ctypes.byref(k)), ctx)
    return {"lambda": lam, "factors": fs, "phi_prev": ph, "outer_done": k.value}


def cpapr_set_state(ctx, state: dict) -> None:
    lam = _as_f64(state["lambda"])
    fs = [_as_f64(A) for A in state["factors"]]
    arr_f = (ctypes.c_void_p * len(fs))(*[_ptr(A) for A in fs])
    ph = state.get("phi_prev")
    arr_p = None
    if ph is not None:
        ph = [_as_f64(A) for A in ph]
        arr_p = (ctypes.c_void_p * len(ph))(*[_ptr(A) for A in ph])
    _check(load().cpapr_set_state(ctx, _ptr(lam), arr_f, arr_p, int(state.get("outer_done", 0))), ctx)


def _out_matrix(ctx, mode, out):
    if out is not None:
        return out
    info = cpapr_get_info(ctx)
    return np.zeros((info.dims[mode], info.rank))


def cpapr_phi(ctx, mode: int, B=None, out=None):
    out = _out_matrix(ctx, mode, out)
    Bc = _as_f64(B) if B is not None else None
    _check(load().cpapr_phi(ctx, int(mode), _ptr(Bc), _ptr(out)), ctx)
    return out


def cpapr_phi_noalloc(ctx, mode: int, out, B=None):
    """Phi^(mode) into the device buffer `out` (I_mode x R float64, e.g. a CUDA
    torch tensor) without any device allocation inside the call: the kernel's
    scratch comes from a fixed array the library carries on every GPU.  For
    callers that cannot let the library call cudaMalloc (memory owned by
    another allocator, loops that must not block on allocation).  B, if
    given, is a device buffer too.  Overlapping calls share that scratch and
    race; make the first call on a device before any stream capture."""
    _check(load().cpapr_phi_noalloc(ctx, int(mode), _ptr(B), _ptr(out)), ctx)
    return out


def cpapr_mttkrp(ctx, mode: int, out=None):
    out = _out_matrix(ctx, mode, out)
    _check(load().cpapr_mttkrp(ctx, int(mode), _ptr(out)), ctx)
    return out


def cpapr_loglik(ctx) -> float:
    v = ctypes.c_double()
    _check(load().cpapr_loglik(ctx, ctypes.byref(v)), ctx)
    return v.value


def cpapr_mu_solve(ctx, tol=1e-4, max_outer=10, max_inner=10, trace=False, ll_trace=None) -> dict:
    """trace: also return the inner iterations per (outer, mode), the KKT
    violation of every outer iteration and, unless ll_trace is False, the
    log-likelihood after every outer iteration."""
    if ll_trace is None:
        ll_trace = trace
    res = Result()
    info = cpapr_get_info(ctx) if trace else None
    inner = np.zeros(max(max_outer, 1) * (info.nmodes if info else 1), dtype=np.int32) if trace else None
    kkt = np.zeros(max(max_outer, 1)) if trace else None
    ll = np.zeros(max(max_outer, 1)) if ll_trace else None
    _check(load().cpapr_mu_solve(ctx, float(tol), int(max_outer), int(max_inner), ctypes.byref(res), _ptr(inner),
                                 _ptr(ll), _ptr(kkt)), ctx)
    out = res.as_dict()
    k = res.outer_iters
    if trace:
        out["inner"] = inner[:k * info.nmodes].reshape(k, info.nmodes)
        out["kkt_trace"] = kkt[:k]
    if ll_trace:
        out["loglik_trace"] = ll[:k]
    return out


def cpapr_batch_mu_solve(ctxs, tol=1e-4, max_outer=10, max_inner=10) -> list:
    n = len(ctxs)
    arr = (ctypes.c_void_p * max(n, 1))(*ctxs)
    res = (Result * max(n, 1))()
    _check(load().cpapr_batch_mu_solve(arr, n, float(tol), int(max_outer), int(max_inner), res), None)
    return [res[i].as_dict() for i in range(n)]


def cpapr_kernel_stats(ctx, kind: int, reset: bool = False):
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(load().cpapr_kernel_stats(ctx, int(kind), ctypes.byref(n), ctypes.byref(ms), int(reset)), ctx)
    return n.value, ms.value


def cpapr_last_error(ctx=None) -> str:
    return load().cpapr_last_error(ctx).decode()


def cpapr_version() -> str:
    return load().cpapr_version().decode()


class Tensor:
    """A sparse count tensor resident on the GPU with its CP-APR model."""

    def __init__(self, dims, idx, vals, rank: int, **options):
        self.opt = cpapr_default_options(**options)
        self.ctx = cpapr_create(dims, idx, vals, rank, self.opt)
        self.dims = tuple(int(d) for d in dims)
        self.rank = int(rank)

    def close(self):
        if getattr(self, "ctx", None):
            cpapr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_model(self, lam, factors):
        cpapr_set_model(self.ctx, lam, factors)

    def init_random(self, seed: int):
        cpapr_init_random(self.ctx, seed)

    def get_model(self):
        return cpapr_get_model(self.ctx)

    def phi(self, mode: int, B=None, out=None):
        return cpapr_phi(self.ctx, mode, B, out)

    def mttkrp(self, mode: int, out=None):
        return cpapr_mttkrp(self.ctx, mode, out)

    def loglik(self) -> float:
        return cpapr_loglik(self.ctx)

    def mu_solve(self, tol=1e-4, max_outer=10, max_inner=10, trace=False, ll_trace=None) -> dict:
        return cpapr_mu_solve(self.ctx, tol, max_outer, max_inner, trace, ll_trace)

    def info(self) -> Info:
        return cpapr_get_info(self.ctx)

    def kernel_stats(self, kind: int, reset: bool = False):
        return cpapr_kernel_stats(self.ctx, kind, reset)
