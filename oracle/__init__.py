"""FP64 CPU oracle for CP-APR MU (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The CUDA library never loads it; it shares no
code with the GPU path.  ``cpapr_oracle.c`` holds the arithmetic; this module
compiles it with gcc (IEEE semantics, no FMA contraction, so x86 and Arm give
the same bits) and wraps it with ctypes.

Functions follow the paper (arXiv 2307.03276):
  phi      -- Algorithm 2 evaluated per nonzero as in Algorithm 3
  phi_threads -- the same on several host threads (the CPU baseline's timing)
  mttkrp   -- the unit-denominator variant (Experiment 8, MTTKRP)
  loglik   -- Poisson log-likelihood of the Kruskal model (not in the paper)
  mu_solve -- Algorithm 1 with the readings listed in cpapr_oracle.c
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpapr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

EPS = 1e-10
KAPPA = 0.01
KAPPA_TOL = 1e-10


def build(force: bool = False) -> str:
    """Compiles liboracle.so next to the source (no-op when up to date)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_phi.argtypes = [i32, P, i64, P, P, i32, P, P, i32, f64, i32, P]
        lib.oracle_phi.restype = i32
        lib.oracle_phi_threads.argtypes = [i32, P, i64, P, P, i32, P, P, i32, f64, i32, P, i32]
        lib.oracle_phi_threads.restype = i32
        lib.oracle_loglik.argtypes = [i32, P, i64, P, P, i32, P, P]
        lib.oracle_loglik.restype = f64
        lib.oracle_mu_solve.argtypes = [i32, P, i64, P, P, i32, P, P, f64, i32, i32, f64, f64, f64,
                                        P, P, P, P, P, P]
        lib.oracle_mu_solve.restype = i32
        lib.oracle_init_random.argtypes = [i32, P, i32, ctypes.c_uint64, P, P]
        lib.oracle_init_random.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _ptr_array(mats):
    arr = (ctypes.c_void_p * len(mats))()
    for k, m in enumerate(mats):
        arr[k] = m.ctypes.data
    return arr


def _coo(dims, idx, vals):
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    if idx.ndim != 2 or idx.shape[0] != dims.shape[0] or idx.shape[1] != vals.shape[0]:
        raise ValueError("idx must be [N, nnz] and vals [nnz]")
    return dims, idx, vals


def _factors(factors, dims, R):
    out = []
    for m, A in enumerate(factors):
        A = np.ascontiguousarray(A, dtype=np.float64)
        if A.shape != (int(dims[m]), R):
            raise ValueError(f"factor {m} must be {int(dims[m])}x{R}")
        out.append(A)
    return out


def phi(dims, idx, vals, factors, B, mode: int, eps: float = EPS) -> np.ndarray:
    """Phi^(mode) = (X_(n) ./ max(B Pi, eps)) Pi^T, one nonzero at a time."""
    return _phi_or_mttkrp(dims, idx, vals, factors, B, mode, eps, 0)


def mttkrp(dims, idx, vals, factors, mode: int) -> np.ndarray:
    """X_(n) times the Khatri-Rao product of the other factors."""
    R = np.asarray(factors[0]).shape[1]
    B = np.zeros((int(dims[mode]), R))
    return _phi_or_mttkrp(dims, idx, vals, factors, B, mode, EPS, 1)


def _phi_or_mttkrp(dims, idx, vals, factors, B, mode, eps, unit):
    lib = _load()
    dims, idx, vals = _coo(dims, idx, vals)
    R = np.asarray(factors[0]).shape[1]
    fs = _factors(factors, dims, R)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.shape != (int(dims[mode]), R):
        raise ValueError("B must be I_n x R")
    out = np.zeros((int(dims[mode]), R))
    rc = lib.oracle_phi(len(dims), _ptr(dims), vals.shape[0], _ptr(idx), _ptr(vals), R, _ptr_array(fs),
                        _ptr(B), int(mode), float(eps), int(unit), _ptr(out))
    if rc != 0:
        raise ValueError(f"oracle_phi failed with code {rc}")
    return out


def phi_threads(dims, idx, vals, factors, B, mode: int, nthreads: int, eps: float = EPS) -> np.ndarray:
    """The same Phi^(mode) on `nthreads` host threads, each owning a range of
    rows of Phi (about nnz / nthreads nonzeros each) and summing them exactly
    as phi() does: the CPU baseline on all cores.  Bit-for-bit equal to phi()."""
    lib = _load()
    dims, idx, vals = _coo(dims, idx, vals)
    R = np.asarray(factors[0]).shape[1]
    fs = _factors(factors, dims, R)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if B.shape != (int(dims[mode]), R):
        raise ValueError("B must be I_n x R")
    out = np.zeros((int(dims[mode]), R))
    rc = lib.oracle_phi_threads(len(dims), _ptr(dims), vals.shape[0], _ptr(idx), _ptr(vals), R, _ptr_array(fs),
                                _ptr(B), int(mode), float(eps), 0, _ptr(out), int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle_phi_threads failed with code {rc}")
    return out


def loglik(dims, idx, vals, lam, factors) -> float:
    lib = _load()
    dims, idx, vals = _coo(dims, idx, vals)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    fs = _factors(factors, dims, lam.shape[0])
    return float(lib.oracle_loglik(len(dims), _ptr(dims), vals.shape[0], _ptr(idx), _ptr(vals), lam.shape[0],
                                   _ptr(lam), _ptr_array(fs)))


def mu_solve(dims, idx, vals, lam, factors, tol=1e-4, max_outer=10, max_inner=10, eps=EPS, kappa=KAPPA,
             kappa_tol=KAPPA_TOL) -> dict:
    """Algorithm 1 from the given model; returns the final model and traces."""
    lib = _load()
    dims, idx, vals = _coo(dims, idx, vals)
    lam = np.array(lam, dtype=np.float64)
    R = lam.shape[0]
    fs = [np.array(A, dtype=np.float64) for A in _factors(factors, dims, R)]
    N = len(dims)
    outer = ctypes.c_int(0)
    inner = ctypes.c_int(0)
    conv = ctypes.c_int(0)
    ll = np.full(max(max_outer, 1), np.nan)
    kkt = np.full(max(max_outer, 1), np.nan)
    itr = np.zeros(max(max_outer, 1) * N, dtype=np.int32)
    rc = lib.oracle_mu_solve(N, _ptr(dims), vals.shape[0], _ptr(idx), _ptr(vals), R, _ptr(lam), _ptr_array(fs),
                             float(tol), int(max_outer), int(max_inner), float(eps), float(kappa),
                             float(kappa_tol), ctypes.byref(outer), ctypes.byref(inner), ctypes.byref(conv),
                             _ptr(ll), _ptr(kkt), _ptr(itr))
    if rc != 0:
        raise ValueError(f"oracle_mu_solve failed with code {rc}")
    k = outer.value
    return {"lambda": lam, "factors": fs, "outer_iters": k, "total_inner": inner.value,
            "converged": bool(conv.value), "loglik": ll[:k].copy(), "kkt": kkt[:k].copy(),
            "inner": itr[:k * N].reshape(k, N).copy()}


def init_random(dims, rank: int, seed: int):
    """U(0,1) factors from SplitMix64, columns scaled to sum 1, lambda = products of the sums."""
    lib = _load()
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    lam = np.zeros(rank)
    fs = [np.zeros((int(d), rank)) for d in dims]
    rc = lib.oracle_init_random(len(dims), _ptr(dims), rank, ctypes.c_uint64(seed), _ptr(lam), _ptr_array(fs))
    if rc != 0:
        raise ValueError(f"oracle_init_random failed with code {rc}")
    return lam, fs
