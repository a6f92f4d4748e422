"""libcg Python binding: argument marshalling over the C ABI of ``include/libcg.h``.

Every step of the solver runs in the CUDA kernels of ``libcg.so``; this module
only passes device pointers of torch tensors, sizes and the current CUDA
stream.  There is no CPU fallback: if ``libcg.so`` cannot be loaded, importing
the functions raises.

The functions keep the C names (``cg_create``, ``cg_spmv``, ``cg_solve`` ...).
Paper anchors: CSR SpMV, Sec. 3.1; CG iteration, Alg. 1; fused kernels, Sec. 3.3.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

CG_OK, CG_NOT_CONVERGED = 0, 1
CG_ERR_INVALID, CG_ERR_BREAKDOWN, CG_ERR_NUMERIC = -1, -2, -3
CG_ERR_TIMEOUT, CG_ERR_CUDA, CG_ERR_OOM = -4, -5, -6
CG_PRECOND_NONE, CG_PRECOND_JACOBI, CG_PRECOND_FSAI = 0, 1, 2
CG_PREC_FP64, CG_PREC_FP32_IR, CG_PREC_FP32_RU = 0, 1, 2
CG_OPT_MAX_RESTARTS, CG_OPT_BARRIER_TIMEOUT_MS, CG_OPT_GRID_CTAS = 0, 1, 2
CG_OPT_IR_TOL_INNER, CG_OPT_IR_MAX_OUTER, CG_OPT_DEBUG_SKIP_ARRIVAL = 3, 4, 5
CG_OPT_PHASE_TIMERS, CG_OPT_LOOP_MODE = 6, 7

# every symbol include/libcg.h declares
EXPORTS = ("cg_create", "cg_set_stream", "cg_set_option", "cg_spmv", "cg_solve",
           "cg_solve_host", "cg_get_solve_info", "cg_get_matrix_info", "cg_destroy",
           "cg_last_error", "cg_status_string", "cg_solve_noalloc", "cg_batch_create",
           "cg_solve_batch", "cg_batch_get_system", "cg_batch_get_tuning", "cg_fsai_classic",
           "cg_fsai_set_factor", "cg_fsai_get_factor", "cg_fsai_load", "cg_fsai_load_f32",
           "cg_fsai_loss_grad", "cg_adam_step", "cg_prepare", "cg_loop_spmv")
CG_MLP_INPUTS, CG_MLP_HIDDEN, CG_MLP_PARAMS = 32, 64, 6337
CG_NOALLOC_MAX_ROWS = 65536
CG_BATCH_MAX_SYSTEMS = 4096


class CGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("relres_true", ctypes.c_double), ("relres_rec", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("bytes_moved", ctypes.c_int64),
                ("kernel_bytes_per_iter", ctypes.c_int64), ("phase_ms", ctypes.c_double * 6),
                ("loop_form", ctypes.c_int32), ("kernel_launches", ctypes.c_int32),
                ("precond_used", ctypes.c_int32)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_ms"] = list(self.phase_ms)
        return d


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcg.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libcg.so not built at {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    pi32, pf64, pi64 = (ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_int64))
    lib.cg_create.argtypes = [i64, P, P, P, ctypes.POINTER(P)]
    lib.cg_set_stream.argtypes = [P, P]
    lib.cg_set_option.argtypes = [P, i32, f64]
    lib.cg_spmv.argtypes = [P, P, P]
    lib.cg_solve.argtypes = [P, P, P, f64, i32, i32, i32, pi32, pf64]
    lib.cg_solve_host.argtypes = [P, P, P, f64, i32, i32, i32, pi32, pf64]
    lib.cg_get_solve_info.argtypes = [P, ctypes.POINTER(SolveInfo)]
    lib.cg_get_matrix_info.argtypes = [P, pi64, pi64, pi64, pi64, pi32]
    lib.cg_destroy.argtypes = [P]
    lib.cg_destroy.restype = None
    lib.cg_last_error.argtypes = [P]
    lib.cg_last_error.restype = ctypes.c_char_p
    lib.cg_status_string.argtypes = [i32]
    lib.cg_status_string.restype = ctypes.c_char_p
    lib.cg_solve_noalloc.argtypes = [i64, i64, P, P, P, P, P, f64, i32, i32, P, pi32, pf64]
    lib.cg_solve_noalloc.restype = ctypes.c_int
    lib.cg_batch_create.argtypes = [i32, pi64, P, P, P, ctypes.POINTER(P)]
    lib.cg_fsai_classic.argtypes = [P]
    lib.cg_fsai_set_factor.argtypes = [P, P]
    lib.cg_fsai_get_factor.argtypes = [P, P, pi64, pi32]
    lib.cg_fsai_load.argtypes = [P, P, i64]
    lib.cg_fsai_load_f32.argtypes = [P, P, i64]
    lib.cg_prepare.argtypes = [P, i32, i32]
    lib.cg_loop_spmv.argtypes = [P, i32, i32, P, P, i32, pi64]
    lib.cg_fsai_loss_grad.argtypes = [P, P, P, P, i32, f64, pf64]
    f32 = ctypes.c_float
    lib.cg_adam_step.argtypes = [P, P, P, P, i64, f32, f32, f32, f32, i32, P]
    lib.cg_solve_batch.argtypes = [P, P, P, f64, i32, i32, i32, pi32, pf64]
    lib.cg_batch_get_system.argtypes = [P, i32, pi32, pi32, pi32, pf64]
    lib.cg_batch_get_tuning.argtypes = [P, i32, i32, pi32, pi32, pi32, ctypes.POINTER(ctypes.c_float), pi32]
    for name in ("cg_create", "cg_set_stream", "cg_set_option", "cg_spmv", "cg_solve",
                 "cg_solve_host", "cg_get_solve_info", "cg_get_matrix_info", "cg_fsai_load_f32", "cg_prepare",
                 "cg_loop_spmv"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().cg_status_string(int(status)).decode()


def _stream_ptr(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype, name, numel=None):
    """Device pointer of a contiguous CUDA tensor of `dtype` on the current device
    (and of `numel` elements when given); None stays None."""
    import torch
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous CUDA {dtype} tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name}: tensor is on cuda:{t.device.index}, the current device is "
                         f"cuda:{torch.cuda.current_device()}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Handle:
    """Owns a cg_handle; keeps the borrowed CSR tensors alive until destroyed."""

    def __init__(self, ptr, n, keep, batch=False):
        self._ptr = ptr
        self.n = n
        self._keep = keep
        self.batch = batch

    @property
    def vec_len(self):
        """Length single-system vectors must have (None on a batch handle, which the
        library itself refuses for single-system calls)."""
        return None if self.batch else self.n

    @property
    def ptr(self):
        if self._ptr is None:
            raise ValueError("handle already destroyed")
        return self._ptr

    def __del__(self):
        try:
            cg_destroy(self)
        except Exception:
            pass


def cg_create(n: int, rowptr, colind, vals) -> Handle:
    """Create a solver for the CSR matrix (device int32/int32/float64 tensors)."""
    import torch
    lib = load()
    out = ctypes.c_void_p()
    torch.cuda.current_stream().synchronize()
    nnz = colind.numel() if colind is not None else 0
    st = lib.cg_create(int(n), _dptr(rowptr, torch.int32, "rowptr", int(n) + 1),
                       _dptr(colind, torch.int32, "colind"),
                       _dptr(vals, torch.float64, "vals", nnz if vals is not None else None),
                       ctypes.byref(out))
    if st != CG_OK:
        raise CGError(st, lib.cg_last_error(None).decode())
    return Handle(out, int(n), (rowptr, colind, vals))


def cg_last_error(h: Handle | None = None) -> str:
    return load().cg_last_error(None if h is None else h.ptr).decode()


def cg_set_stream(h: Handle, stream=None) -> int:
    return load().cg_set_stream(h.ptr, _stream_ptr(stream))


def cg_set_option(h: Handle, option: int, value: float) -> int:
    return load().cg_set_option(h.ptr, int(option), float(value))


def cg_spmv(h: Handle, x, y) -> int:
    """y = A x on the current stream."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    return lib.cg_spmv(h.ptr, _dptr(x, torch.float64, "x", h.vec_len),
                       _dptr(y, torch.float64, "y", h.vec_len))


def cg_solve(h: Handle, b, x, tol: float = 1e-8, maxit: int = 1000,
             precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64):
    """Solve A x = b on the current stream; x holds x0 on entry.
    Returns (status, iters, relres_true)."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = lib.cg_solve(h.ptr, _dptr(b, torch.float64, "b", h.vec_len),
                      _dptr(x, torch.float64, "x", h.vec_len),
                      float(tol), int(maxit), int(precond), int(precision), ctypes.byref(it),
                      ctypes.byref(rel))
    return st, it.value, rel.value


def cg_solve_host(h: Handle, b_host, x_host, tol: float = 1e-8, maxit: int = 1000,
                  precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64):
    """cg_solve with host (preferably pinned) float64 tensors; copies happen inside
    the call.  Returns (status, iters, relres_true)."""
    import torch
    for t, name in ((b_host, "b_host"), (x_host, "x_host")):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name}: expected a contiguous host float64 tensor")
        if h.vec_len is not None and t.numel() != h.vec_len:
            raise ValueError(f"{name}: expected {h.n} elements, got {t.numel()}")
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = lib.cg_solve_host(h.ptr, ctypes.c_void_p(b_host.data_ptr()),
                           ctypes.c_void_p(x_host.data_ptr()), float(tol), int(maxit),
                           int(precond), int(precision), ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def cg_solve_noalloc(rowptr, colind, vals, b, x, tol: float = 1e-8, maxit: int = 1000,
                     precond: int = CG_PRECOND_JACOBI):
    """Handle-free solve that allocates no device memory (for callers that cannot call
    cudaMalloc); n <= CG_NOALLOC_MAX_ROWS, single CTA, so small systems only.  Runs on
    the current stream; x holds x0 on entry.  Returns (status, iters, relres_true)."""
    import torch
    n = rowptr.numel() - 1
    nnz = colind.numel() if colind is not None else 0
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    st = load().cg_solve_noalloc(n, nnz, _dptr(rowptr, torch.int32, "rowptr"),
                                 _dptr(colind, torch.int32, "colind"),
                                 _dptr(vals, torch.float64, "vals", nnz if vals is not None else None),
                                 _dptr(b, torch.float64, "b", n), _dptr(x, torch.float64, "x", n),
                                 float(tol), int(maxit),
                                 int(precond), _stream_ptr(), ctypes.byref(it), ctypes.byref(rel))
    return st, it.value, rel.value


def cg_prepare(h: Handle, precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64) -> int:
    """Build the loop matrix and work vectors a solve with (precond, precision) needs."""
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    return lib.cg_prepare(h.ptr, int(precond), int(precision))


def cg_loop_spmv(h: Handle, p, q, precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64,
                 reps: int = 1):
    """q = A^ p with the solve loop's SpMV kernel, `reps` launches on the current stream
    (A^ = D^-1/2 A D^-1/2 with Jacobi).  p, q: CUDA float64 (fp64) or float32 (fp32
    precisions) tensors of n elements.  Returns (status, bytes one launch must move)."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    dt = torch.float64 if precision == CG_PREC_FP64 else torch.float32
    nb = ctypes.c_int64(0)
    st = lib.cg_loop_spmv(h.ptr, int(precond), int(precision), _dptr(p, dt, "p", h.vec_len),
                          _dptr(q, dt, "q", h.vec_len), int(reps), ctypes.byref(nb))
    return st, nb.value


def cg_get_solve_info(h: Handle) -> dict:
    info = SolveInfo()
    st = load().cg_get_solve_info(h.ptr, ctypes.byref(info))
    if st != CG_OK:
        raise CGError(st, cg_last_error(h))
    return info.as_dict()


def cg_get_matrix_info(h: Handle) -> dict:
    n, nnz, nrb, nlong = (ctypes.c_int64() for _ in range(4))
    g = ctypes.c_int32()
    load().cg_get_matrix_info(h.ptr, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nrb),
                              ctypes.byref(nlong), ctypes.byref(g))
    return {"n": n.value, "nnz": nnz.value, "row_blocks": nrb.value, "long_rows": nlong.value,
            "grid_ctas": g.value}


def cg_destroy(h: Handle) -> None:
    if h is not None and h._ptr is not None and _lib is not None:
        _lib.cg_destroy(h._ptr)
        h._ptr = None
        h._keep = None


def _ptr_array(tensors, dtype, name):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _dptr(t, dtype, f"{name}[{i}]").value
    return arr


def cg_batch_create(rowptrs, colinds, valss) -> Handle:
    """Create a batch solver for len(rowptrs) systems (lists of device int32 / int32 /
    float64 tensors, one CSR per system)."""
    import torch
    lib = load()
    ns = len(rowptrs)
    if not (len(colinds) == ns and len(valss) == ns):
        raise ValueError("cg_batch_create: rowptrs, colinds and valss differ in length")
    nrows = (ctypes.c_int64 * max(ns, 1))(*[int(r.numel()) - 1 for r in rowptrs])
    rp = _ptr_array(rowptrs, torch.int32, "rowptr")
    ci = _ptr_array(colinds, torch.int32, "colind")
    va = _ptr_array(valss, torch.float64, "vals")
    out = ctypes.c_void_p()
    torch.cuda.current_stream().synchronize()
    st = lib.cg_batch_create(ns, nrows, rp, ci, va, ctypes.byref(out))
    if st != CG_OK:
        raise CGError(st, lib.cg_last_error(None).decode())
    return Handle(out, sum(int(r.numel()) - 1 for r in rowptrs),
                  (list(rowptrs), list(colinds), list(valss)), batch=True)


def cg_solve_batch(h: Handle, bs, xs, tol: float = 1e-8, maxit: int = 1000,
                   precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64):
    """Solve every system of a batch handle on the current stream; xs hold the initial
    guesses on entry.  Returns (status, iters list, relres list)."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    ns = len(bs)
    if len(xs) != ns:
        raise ValueError("cg_solve_batch: bs and xs differ in length")
    its = (ctypes.c_int32 * max(ns, 1))()
    rels = (ctypes.c_double * max(ns, 1))()
    st = lib.cg_solve_batch(h.ptr, _ptr_array(bs, torch.float64, "b"), _ptr_array(xs, torch.float64, "x"),
                            float(tol), int(maxit), int(precond), int(precision), its, rels)
    return st, list(its)[:ns], list(rels)[:ns]


def cg_batch_get_system(h: Handle, s: int) -> dict:
    st, it, rs = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rel = ctypes.c_double()
    r = load().cg_batch_get_system(h.ptr, int(s), ctypes.byref(st), ctypes.byref(it), ctypes.byref(rs),
                                   ctypes.byref(rel))
    if r != CG_OK:
        raise CGError(r, cg_last_error(h))
    return {"status": st.value, "iters": it.value, "restarts": rs.value, "relres": rel.value}


def cg_batch_get_tuning(h: Handle, precond: int = CG_PRECOND_JACOBI, precision: int = CG_PREC_FP64) -> dict:
    cnt, chosen = ctypes.c_int32(), ctypes.c_int32()
    grids = (ctypes.c_int32 * 8)()
    per_sm = (ctypes.c_int32 * 8)()
    ms = (ctypes.c_float * 8)()
    r = load().cg_batch_get_tuning(h.ptr, int(precond), int(precision), ctypes.byref(cnt), grids, per_sm, ms,
                                   ctypes.byref(chosen))
    if r != CG_OK:
        raise CGError(r, cg_last_error(h))
    k = cnt.value
    return {"grids": list(grids)[:k], "ctas_per_sm": list(per_sm)[:k], "ms": list(ms)[:k],
            "chosen": chosen.value}


def cg_fsai_classic(h: Handle) -> int:
    """Build the classic FSAI factor of the handle's matrix (on the current stream)."""
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    return lib.cg_fsai_classic(h.ptr)


def cg_fsai_set_factor(h: Handle, g_tril) -> int:
    """Use the caller's factor: a CUDA float64 tensor of G's values in tril(A) order."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    return lib.cg_fsai_set_factor(h.ptr, _dptr(g_tril, torch.float64, "g_tril"))


def cg_fsai_get_factor(h: Handle):
    """(status, values tensor or None, kind) of the handle's current factor."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    nt, kind = ctypes.c_int64(), ctypes.c_int32()
    st = lib.cg_fsai_get_factor(h.ptr, None, ctypes.byref(nt), ctypes.byref(kind))
    if st != CG_OK or kind.value == 0:
        return st, None, kind.value
    g = torch.empty(nt.value, dtype=torch.float64, device="cuda")
    st = lib.cg_fsai_get_factor(h.ptr, _dptr(g, torch.float64, "g"), None, None)
    return st, g, kind.value


def cg_fsai_load(h: Handle, params) -> int:
    """Compute the handle's FSAI factor with the MLP; params: CG_MLP_PARAMS fp32 values
    (host array or tensor), which the library rounds to bf16 (cg_fsai_load_f32)."""
    import numpy as np
    if hasattr(params, "detach"):
        params = params.detach().cpu().numpy()
    w = np.ascontiguousarray(params, dtype=np.float32)
    if w.size != CG_MLP_PARAMS:
        raise ValueError(f"expected {CG_MLP_PARAMS} parameters")
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    return lib.cg_fsai_load_f32(h.ptr, ctypes.c_void_p(w.ctypes.data), w.size)


def cg_fsai_loss_grad(h: Handle, params, grad, resid=None, lam: float = 0.1):
    """Loss of the MLP on the handle's matrix and its gradient (written into grad).
    params, grad: CUDA float32 tensors of CG_MLP_PARAMS; resid: CUDA float64 [k, n] or
    None.  Returns (status, loss)."""
    import torch
    lib = load()
    lib.cg_set_stream(h.ptr, _stream_ptr())
    loss = ctypes.c_double(0.0)
    k = 0 if resid is None else int(resid.shape[0])
    st = lib.cg_fsai_loss_grad(h.ptr, _dptr(params, torch.float32, "params"), _dptr(grad, torch.float32, "grad"),
                               None if resid is None else _dptr(resid, torch.float64, "resid"), k, float(lam),
                               ctypes.byref(loss))
    return st, loss.value


def cg_adam_step(params, grad, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8) -> int:
    """One Adam step on CUDA float32 tensors (current stream)."""
    import torch
    return load().cg_adam_step(_dptr(params, torch.float32, "params"), _dptr(grad, torch.float32, "grad"),
                               _dptr(m, torch.float32, "m"), _dptr(v, torch.float32, "v"), params.numel(),
                               float(lr), float(beta1), float(beta2), float(eps), int(step), _stream_ptr())


@dataclass
class Result:
    status: int
    iters: int
    relres: float


class Solver:
    """Convenience wrapper: ``Solver(rowptr, colind, vals).solve(b, x)``."""

    def __init__(self, rowptr, colind, vals):
        self.n = rowptr.numel() - 1
        self.h = cg_create(self.n, rowptr, colind, vals)

    def spmv(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        st = cg_spmv(self.h, x, y)
        if st != CG_OK:
            raise CGError(st, cg_last_error(self.h))
        return y

    def solve(self, b, x=None, tol=1e-8, maxit=1000, precond=CG_PRECOND_JACOBI,
              precision=CG_PREC_FP64, check=True) -> Result:
        import torch
        if x is None:
            x = torch.zeros_like(b)
        st, it, rel = cg_solve(self.h, b, x, tol, maxit, precond, precision)
        if check and st < 0:
            raise CGError(st, cg_last_error(self.h))
        return Result(st, it, rel)

    def set_option(self, option, value):
        st = cg_set_option(self.h, option, value)
        if st != CG_OK:
            raise CGError(st, cg_last_error(self.h))

    def info(self):
        return cg_get_solve_info(self.h)

    def close(self):
        cg_destroy(self.h)
