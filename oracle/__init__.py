"""CG oracle — TEST INFRASTRUCTURE ONLY.

Plain sequential fp64 restatement of the sparse CG hot path (``oracle.c``),
used by the tests, the smoke check and the benchmark's CPU-baseline leg to
check the CUDA library.  The product path never imports this package, and this
package imports nothing from the product package.

Citations (the paper: "A Preliminary Study on Simultaneous Coscheduling for
Discrete GPU vs. Fused GPU"): CSR SpMV, Sec. 3.1; CG iteration, Alg. 1;
fp64 throughout, Sec. 3.1; recomputed final residual, Sec. 3.1.  The readings
R1-R8 taken where the paper is silent are listed in ``oracle.c``; the FSAI
preconditioner and its MLP (not in the paper) are in ``oracle.fsai`` (F1-F8).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_lib_omp = None

OK, NOT_CONVERGED, ERR_INVALID, ERR_BREAKDOWN, ERR_NUMERIC, ERR_OOM = 0, 1, -1, -2, -3, -6


def _compile(lib, extra):
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", *extra,
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, lib)


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no FMA contraction, no arch-specific flags); the
    OpenMP build used only to time the oracle on all host cores is attempted too."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_LIB, [])
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        try:
            _compile(_LIB_OMP, ["-fopenmp"])
        except (subprocess.CalledProcessError, OSError):
            pass  # no OpenMP runtime: the all-core timing leg reports itself unavailable
    return _LIB


def openmp():
    """The all-core build of the same oracle (row loops split over OpenMP threads, Sec.
    3.3), for timing only: its reductions sum per thread, so it never checks results.
    Returns (library, threads) or (None, 0) when no OpenMP build exists."""
    global _lib_omp
    if _lib_omp is None:
        build()
        if not os.path.exists(_LIB_OMP):
            return None, 0
        _lib_omp = _bind(ctypes.CDLL(_LIB_OMP))
    return _lib_omp, int(_lib_omp.or_threads())


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("relres_rec", ctypes.c_double), ("relres_true", ctypes.c_double)]


def _bind(lib):
    """Declare the C signatures on a loaded oracle library and return it."""
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.or_spmv.argtypes = [i64, P, P, P, P, P]
    lib.or_spmv.restype = None
    lib.or_dot.argtypes = [i64, P, P]
    lib.or_dot.restype = f64
    lib.or_true_relres.argtypes = [i64, P, P, P, P, P]
    lib.or_true_relres.restype = f64
    lib.or_jacobi_dinv.argtypes = [i64, P, P, P, P]
    lib.or_jacobi_dinv.restype = ctypes.c_int
    lib.or_pcg.argtypes = [i64, P, P, P, P, P, f64, i32, i32, i32, P, i32, P,
                           ctypes.POINTER(_Result)]
    lib.or_pcg.restype = ctypes.c_int
    lib.or_pcg_ir.argtypes = [i64, P, P, P, P, P, f64, f64, i32, i32, i32, P,
                              ctypes.POINTER(_Result)]
    lib.or_pcg_ir.restype = ctypes.c_int
    lib.or_pcg_ru.argtypes = lib.or_pcg_ir.argtypes
    lib.or_pcg_ru.restype = ctypes.c_int
    lib.or_threads.argtypes = []
    lib.or_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _csr(A):
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = np.ascontiguousarray(A.vals, dtype=np.float64)
    return A.n, rp, ci, va


@dataclass
class Solve:
    x: np.ndarray
    status: int
    iters: int
    restarts: int
    relres_rec: float
    relres_true: float
    res_hist: np.ndarray | None = None
    p_hist: np.ndarray | None = None
    outer_hist: np.ndarray | None = None


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x in fp64, each row summed in storage order (Sec. 3.1)."""
    n, rp, ci, va = _csr(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n, dtype=np.float64)
    _load().or_spmv(n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def true_relres(A, b: np.ndarray, x: np.ndarray) -> float:
    """||b - A x|| / ||b|| in fp64 (Sec. 3.1, recomputed residual)."""
    n, rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().or_true_relres(n, _p(rp), _p(ci), _p(va), _p(b), _p(x)))


def jacobi_dinv(A) -> np.ndarray:
    n, rp, ci, va = _csr(A)
    d = np.empty(n, dtype=np.float64)
    if _load().or_jacobi_dinv(n, _p(rp), _p(ci), _p(va), _p(d)) != 0:
        raise ValueError("matrix has a missing or non-positive diagonal")
    return d


def pcg(A, b, x0=None, tol=1e-8, maxit=1000, precond=1, max_restarts=3,
        p_hist_k=0, res_hist=False, lib=None) -> Solve:
    """(Jacobi-preconditioned) CG, Alg. 1 with readings R1-R5 (see oracle.c).

    precond: 0 = none (the paper's unpreconditioned CG), 1 = Jacobi.  lib: another build
    of the oracle (openmp()[0], for timing on all cores); default the checker build."""
    n, rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    ph = np.zeros((p_hist_k, n)) if p_hist_k else None
    rh = np.full(maxit + 1, np.nan) if res_hist else None
    res = _Result()
    (lib or _load()).or_pcg(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, maxit, precond,
                   max_restarts, _p(ph), p_hist_k, _p(rh), ctypes.byref(res))
    if rh is not None:
        rh = rh[: res.iters + 1]
    return Solve(x, res.status, res.iters, res.restarts, res.relres_rec, res.relres_true,
                 rh, ph)


def pcg_ir(A, b, x0=None, tol=1e-10, tol_in=1e-4, maxit=100000, max_outer=30,
           precond=1) -> Solve:
    """fp32-inner / fp64-outer iterative refinement (reading R6).  iters = total
    inner iterations, restarts = refinement steps."""
    n, rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    oh = np.full(max_outer + 1, np.nan)
    res = _Result()
    _load().or_pcg_ir(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, tol_in, maxit,
                      max_outer, precond, _p(oh), ctypes.byref(res))
    return Solve(x, res.status, res.iters, res.restarts, res.relres_rec, res.relres_true,
                 outer_hist=oh[: res.restarts + 1])


def pcg_ru(A, b, x0=None, tol=1e-10, tol_in=1e-4, maxit=100000, max_updates=30,
           precond=1) -> Solve:
    """fp32 inner PCG with fp64 reliable updates (reading R8): the refinement of R6 with
    the search direction carried over each update.  iters = total inner iterations,
    restarts = fp64 updates."""
    n, rp, ci, va = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    oh = np.full(max_updates + 1, np.nan)
    res = _Result()
    _load().or_pcg_ru(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, tol_in, maxit,
                      max_updates, precond, _p(oh), ctypes.byref(res))
    return Solve(x, res.status, res.iters, res.restarts, res.relres_rec, res.relres_true,
                 outer_hist=oh[: res.restarts + 1])
