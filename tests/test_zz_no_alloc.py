"""The allocation-free entry point, cg_solve_noalloc, against the handle-based cg_solve.

cg_solve_noalloc is for callers that cannot allocate device memory (a plugin inside a
framework that owns all device memory through its own pool, code that may not hold
allocations of its own, a loop where cudaMalloc could stall the device).  Its scratch is
a fixed device array shared by every call, so the test makes two calls in a row on
different systems and then repeats the first: each answer must agree with cg_solve within
the tolerances of the parity tests, and a repeat must reproduce the first call exactly.
This file is collected last so that a failure here cannot hide another test's result.
"""
import math

import numpy as np
import pytest

import cgproblems as gen
import oracle
from helpers import to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402


def handle_solve(A, b, tol, maxit, precond):
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, xd, tol, maxit, precond, cg.CG_PREC_FP64)
    x = xd.cpu().numpy()
    cg.cg_destroy(h)
    return st, it, rel, x


def noalloc_solve(A, b, tol, maxit, precond):
    rp, ci, va = to_device(A)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve_noalloc(rp, ci, va, bd, xd, tol, maxit, precond)
    torch.cuda.synchronize()
    return st, it, rel, xd.cpu().numpy()


def check_agrees(A, b, tol, maxit, precond):
    st0, it0, rel0, x0 = handle_solve(A, b, tol, maxit, precond)
    st1, it1, rel1, x1 = noalloc_solve(A, b, tol, maxit, precond)
    assert st1 == st0 == cg.CG_OK, cg.status_string(st1)
    assert abs(it1 - it0) <= max(3, math.ceil(0.02 * it0)), (it1, it0)
    assert rel1 <= tol and oracle.true_relres(A, b, x1) <= tol * (1 + 1e-6)
    assert np.linalg.norm(x1 - x0) <= 1e-4 * np.linalg.norm(x0)
    return st1, it1, rel1, x1


def test_noalloc_matches_cg_solve_on_consecutive_calls():
    A1 = gen.lap2d(48, 9, 0.05)                 # Jacobi, 2304 rows
    b1 = oracle.spmv(A1, gen.xstar(A1.n, 1))
    A2 = gen.lap3d7(40)                         # plain CG, 64000 rows (near the limit)
    b2 = oracle.spmv(A2, gen.xstar(A2.n, 2))
    first = check_agrees(A1, b1, 1e-8, 5000, cg.CG_PRECOND_JACOBI)
    check_agrees(A2, b2, 1e-8, 5000, cg.CG_PRECOND_NONE)
    again = noalloc_solve(A1, b1, 1e-8, 5000, cg.CG_PRECOND_JACOBI)
    assert again[:3] == first[:3] and np.array_equal(again[3], first[3])


def test_noalloc_rejects_more_rows_than_its_scratch_holds():
    lib = cg.load()
    n = cg.CG_NOALLOC_MAX_ROWS + 1
    assert lib.cg_solve_noalloc(n, 0, None, None, None, None, None, 1e-8, 10, 0, None, None,
                                None) == cg.CG_ERR_INVALID


def raw_noalloc(n, nnz, rp, ci, va, b, x, precond):
    """The C entry point itself, with the nnz the caller states (the binding would
    take it from colind's length)."""
    lib = cg.load()
    it = cg.ctypes.c_int32(-1)
    rel = cg.ctypes.c_double(-1.0)
    st = lib.cg_solve_noalloc(n, nnz, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), b.data_ptr(),
                              x.data_ptr(), 1e-8, 500, precond,
                              cg.ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                              cg.ctypes.byref(it), cg.ctypes.byref(rel))
    torch.cuda.synchronize()
    return st


@pytest.mark.parametrize("fault", ["colind_equals_n", "rowptr_end_differs_from_nnz",
                                   "jacobi_zero_diagonal"])
def test_noalloc_refuses_a_malformed_csr_on_the_device_then_recovers(fault):
    """The kernel checks the CSR before any indexed read (rowptr[0] = 0, rowptr[n] = nnz,
    rows non-decreasing, colind in [0, n), a positive diagonal for Jacobi), so each of
    these inputs is refused with CG_ERR_INVALID without touching memory outside the
    buffers.  A valid solve right after must still agree with cg_solve: the shared
    scratch and its result block carry nothing over from the refused call."""
    A = gen.lap2d(24)
    rp, ci, va = (t.clone() for t in to_device(A))
    nnz = A.nnz
    precond = cg.CG_PRECOND_NONE
    if fault == "colind_equals_n":
        ci[nnz // 2] = A.n
    elif fault == "rowptr_end_differs_from_nnz":
        nnz -= 1                       # the buffers keep their full length
    else:
        va[rp[5].item():rp[6].item()] = torch.where(ci[rp[5].item():rp[6].item()] == 5, 0.0,
                                                    va[rp[5].item():rp[6].item()])
        precond = cg.CG_PRECOND_JACOBI
    b = torch.from_numpy(oracle.spmv(A, gen.xstar(A.n, 4))).cuda()
    x = torch.zeros_like(b)
    assert raw_noalloc(A.n, nnz, rp, ci, va, b, x, precond) == cg.CG_ERR_INVALID
    B = gen.lap2d(30, 9, 0.2)
    bb = oracle.spmv(B, gen.xstar(B.n, 5))
    check_agrees(B, bb, 1e-8, 5000, cg.CG_PRECOND_JACOBI)
