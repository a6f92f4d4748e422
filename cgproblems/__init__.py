"""Seeded synthetic SPD problems in CSR form, shared by the oracle and the GPU path.

The builders live in ``gen.c`` (compiled with gcc into ``libcggen.so`` next to
this file); this module only allocates numpy arrays and calls them.  Nothing
here performs conjugate-gradient arithmetic: right-hand sides ``b = A x*`` are
formed by the side that consumes the matrix.

Workload recipes (the paper measures on SuiteSparse matrices, Sec. 4.1, which
are not reproduced; these synthetic families stand in for them):

* ``lap2d(N, 5)``      2-D 5-point Dirichlet Laplacian, stencil (4, -1).
* ``lap3d7(N)``        3-D 7-point Dirichlet Laplacian, stencil (6, -1).
* ``diff3d27(N, s)``   3-D 27-point graph Laplacian, per-edge lognormal weights.
* ``lap2d(N, p, eps)`` anisotropic 5-/9-point 2-D Laplacians (batched solves).
* ``q1aniso(...)``     rotated-anisotropy Q1 finite elements (learned FSAI).
* ``graph_spd(n)``     general sparse SPD: graph Laplacian with power-law degrees.
* ``xstar(n, seed)``   exact solution, uniform in [-1, 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libcggen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libcggen.so (gcc, portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        P = ctypes.c_void_p
        pi64 = ctypes.POINTER(ctypes.c_int64)
        lib.gen_splitmix64.argtypes = [u64, u64]
        lib.gen_splitmix64.restype = u64
        lib.gen_normal.argtypes = [u64, u64]
        lib.gen_normal.restype = f64
        lib.gen_uniform_pm1.argtypes = [i64, u64, P]
        lib.gen_lap2d_size.argtypes = [i64, i32, f64, pi64, pi64]
        lib.gen_lap2d_fill.argtypes = [i64, i32, f64, P, P, P]
        lib.gen_lap3d7_size.argtypes = [i64, pi64, pi64]
        lib.gen_lap3d7_fill.argtypes = [i64, P, P, P]
        lib.gen_diff3d27_size.argtypes = [i64, pi64, pi64]
        lib.gen_diff3d27_fill.argtypes = [i64, f64, u64, P, P, P]
        lib.gen_q1aniso_size.argtypes = [i64, pi64, pi64]
        lib.gen_q1aniso_fill.argtypes = [i64, f64, f64, f64, u64, P, P, P]
        lib.gen_graph_spd_size.argtypes = [i64, i32, u64, pi64, pi64]
        lib.gen_graph_spd_fill.argtypes = [i64, i32, u64, P, P, P]
        for name in ("gen_uniform_pm1", "gen_lap2d_size", "gen_lap2d_fill", "gen_lap3d7_size",
                     "gen_lap3d7_fill", "gen_diff3d27_size", "gen_diff3d27_fill",
                     "gen_q1aniso_size", "gen_q1aniso_fill", "gen_graph_spd_size",
                     "gen_graph_spd_fill"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class CSR:
    """Host CSR matrix: rowptr int32[n+1], colind int32[nnz], vals float64[nnz]."""
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    vals: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.vals, self.colind, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                d[i, self.colind[k]] += self.vals[k]
        return d


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _build(size_fn, fill_fn, size_args, fill_args, name) -> CSR:
    lib = _load()
    n = ctypes.c_int64()
    nnz = ctypes.c_int64()
    if getattr(lib, size_fn)(*size_args, ctypes.byref(n), ctypes.byref(nnz)) != 0:
        raise ValueError(f"{name}: bad arguments {size_args}")
    rowptr = np.empty(n.value + 1, dtype=np.int32)
    colind = np.empty(nnz.value, dtype=np.int32)
    vals = np.empty(nnz.value, dtype=np.float64)
    if getattr(lib, fill_fn)(*fill_args, _ptr(rowptr), _ptr(colind), _ptr(vals)) != 0:
        raise ValueError(f"{name}: fill failed")
    return CSR(n.value, rowptr, colind, vals, name)


def lap2d(N: int, points: int = 5, eps: float = 1.0) -> CSR:
    """2-D anisotropic graph Laplacian on an N x N grid (couplings eps along x, 1 along y;
    the 9-point form adds diagonal couplings (1+eps)/4)."""
    return _build("gen_lap2d_size", "gen_lap2d_fill", (N, points, float(eps)),
                  (N, points, float(eps)), f"lap2d{points}_N{N}_eps{eps:g}")


def lap3d7(N: int) -> CSR:
    """3-D 7-point Dirichlet Laplacian on an N^3 grid."""
    return _build("gen_lap3d7_size", "gen_lap3d7_fill", (N,), (N,), f"lap3d7_N{N}")


def diff3d27(N: int, sigma: float = 1.0, seed: int = 0) -> CSR:
    """3-D 27-point variable-coefficient graph Laplacian, lognormal(0, sigma) edge weights."""
    return _build("gen_diff3d27_size", "gen_diff3d27_fill", (N,), (N, float(sigma), seed),
                  f"diff3d27_N{N}_s{sigma:g}_seed{seed}")


def q1aniso(s: int, sigma_a: float, theta: float, eps: float, seed: int) -> CSR:
    """Q1 rotated-anisotropy diffusion on an s x s interior node grid."""
    return _build("gen_q1aniso_size", "gen_q1aniso_fill", (s,),
                  (s, float(sigma_a), float(theta), float(eps), seed),
                  f"q1aniso_s{s}_seed{seed}")


def graph_spd(n: int, dmax: int = 600, seed: int = 0) -> CSR:
    """General sparse SPD matrix (no stencil structure): a weighted graph Laplacian with
    power-law degrees (a row emits up to dmax/2 couplings, most rows have 2-6 neighbours, a
    few hundred), 70 % of the couplings within 64 rows and 30 % to uniformly random rows,
    diagonal (1 + s_i) times the row's coupling sum with s_i log-uniform in [1e-4, 1e-3]
    (1 for a row without couplings)."""
    return _build("gen_graph_spd_size", "gen_graph_spd_fill", (n, dmax, seed), (n, dmax, seed),
                  f"graph_spd_n{n}_d{dmax}_seed{seed}")


def xstar(n: int, seed: int) -> np.ndarray:
    """Exact solution x*, uniform in [-1, 1) from the counter-based stream `seed`."""
    out = np.empty(n, dtype=np.float64)
    if _load().gen_uniform_pm1(n, seed, _ptr(out)) != 0:
        raise ValueError("xstar: bad arguments")
    return out


def splitmix64(seed: int, ctr: int) -> int:
    return int(_load().gen_splitmix64(seed, ctr))


def normal(seed: int, ctr: int) -> float:
    return float(_load().gen_normal(seed, ctr))


def uniform01(seed: int, ctr: int) -> float:
    """The [0, 1) uniform the builders use for counter `ctr` (53 random bits)."""
    return (splitmix64(seed, ctr) >> 11) * 2.0 ** -53


# --- named workloads -------------------------------------------------------

def batch_members(count: int = 512, seed: int = 0, side_lo: int = 32, side_hi: int = 512):
    """Parameters of a batch of uneven anisotropic 2-D systems: side uniform in
    [side_lo, side_hi], 5- or 9-point alternating by index, eps log-uniform in
    [1e-3, 1].  Returns a list of (side, points, eps)."""
    out = []
    for i in range(count):
        s = seed ^ (0x5EED0000 + i)
        side = side_lo + splitmix64(s, 0) % (side_hi - side_lo + 1)
        points = 5 if i % 2 == 0 else 9
        eps = 10.0 ** (-3.0 * uniform01(s, 1))
        out.append((int(side), points, float(eps)))
    return out


def q1_params(index: int, seed: int = 0, side_lo: int = 256, side_hi: int = 1024):
    """Parameters of matrix `index` of the rotated-anisotropy family: side uniform in
    [side_lo, side_hi], theta uniform in [0, pi), eps log-uniform in [1e-3, 1];
    returns (side, theta, eps, matrix_seed)."""
    s = seed ^ (0xF5A10000 + index)
    side = side_lo + splitmix64(s, 0) % (side_hi - side_lo + 1)
    theta = 3.141592653589793 * uniform01(s, 1)
    eps = 10.0 ** (-3.0 * uniform01(s, 2))
    return int(side), float(theta), float(eps), int(splitmix64(s, 3) >> 1)
