"""The solve loop's own SpMV kernel (cg_loop_spmv) against the plain definition of the
operator it applies, and cg_prepare against the lazy setup of cg_solve.

The loop iterates on A^ = D^-1/2 A D^-1/2 with Jacobi (unit diagonal, Sec. 3.1 SpMV on
the scaled matrix; the iteration is the same as Jacobi-PCG on A) and on A otherwise.
Reference: q_i = p_i + sum_{j != i} A_ij / (sqrt(A_ii) sqrt(A_jj)) p_j (Jacobi) or
q = A p, evaluated in fp64 with numpy on the CPU.  Tolerances from the arithmetic: the
kernel rounds each scaled entry (two products) and sums at most ~30 terms with fused
multiply-adds, so |q - q_ref|_i <= 1e-13 (|A^| |p|)_i in fp64; in fp32 the entries and
the sum are rounded to 24 bits, so the bound is 4e-6 (|A^| |p|)_i.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import cgproblems as gen
import oracle
from helpers import hub_graph_spd, random_graph_spd, spd_from_pattern, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402


def reference(A, p, jac):
    S = A.to_scipy().tocsr()
    if not jac:
        return S @ p, abs(S) @ np.abs(p)
    d = S.diagonal()
    s = 1.0 / np.sqrt(d)
    off = S - sp.diags(d)
    Ah = (off.multiply(s[:, None]).multiply(s[None, :])).tocsr()
    return p + Ah @ p, np.abs(p) + abs(Ah) @ np.abs(p)


MATS = [
    ("lap3d7_23", lambda: gen.lap3d7(23)),                 # diagonal layout, 6 offsets
    ("diff27_14", lambda: gen.diff3d27(14, 1.0, 3)),      # diagonal layout, 26 offsets
    ("q1_45", lambda: gen.q1aniso(45, 1.5, 0.3, 0.05, 2)),  # diagonal layout, 8 offsets
    ("graph_5000", lambda: random_graph_spd(5000, 2, 3)),   # uniform sliced ELL
    ("pattern_long", lambda: spd_from_pattern(6000, 5, long_rows=[(3, 400), (4100, 900)])),
    ("powerlaw_20000", lambda: gen.graph_spd(20000, 600, 1)),   # row-block CSR layout, bulk-staged blocks
    ("powerlaw_hub", lambda: hub_graph_spd(20000, 2, 3000)),    # ... and a row past the block cap
]


@pytest.mark.parametrize("precision", [cg.CG_PREC_FP64, cg.CG_PREC_FP32_RU], ids=["fp64", "fp32"])
@pytest.mark.parametrize("precond", [cg.CG_PRECOND_JACOBI, cg.CG_PRECOND_NONE], ids=["jacobi", "none"])
@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_loop_spmv_matches_the_operator(name, make, precond, precision):
    A = make()
    h = cg.cg_create(A.n, *to_device(A))
    fp64 = precision == cg.CG_PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    p = gen.xstar(A.n, 7)
    if not fp64:
        p = p.astype(np.float32).astype(np.float64)
    pd = torch.from_numpy(p).to(dt).cuda()
    qd = torch.full_like(pd, float("nan"))
    st, nbytes = cg.cg_loop_spmv(h, pd, qd, precond, precision, reps=3)
    assert st == cg.CG_OK, cg.cg_last_error(h)
    torch.cuda.synchronize()
    q = qd.cpu().numpy().astype(np.float64)
    ref, scale = reference(A, p, precond == cg.CG_PRECOND_JACOBI)
    bound = (1e-13 if fp64 else 4e-6) * scale + 1e-300
    assert np.all(np.abs(q - ref) <= bound), np.max(np.abs(q - ref) / bound)
    assert nbytes >= (8 if fp64 else 4) * (A.nnz - A.n) + 2 * (8 if fp64 else 4) * A.n
    cg.cg_destroy(h)


def test_prepare_then_solve_equals_lazy_setup():
    A = gen.lap2d(70, 9, 0.02)
    b = oracle.spmv(A, gen.xstar(A.n, 3))
    out = []
    for prepare in (False, True):
        h = cg.cg_create(A.n, *to_device(A))
        if prepare:
            for prec in (cg.CG_PREC_FP64, cg.CG_PREC_FP32_RU):
                assert cg.cg_prepare(h, cg.CG_PRECOND_JACOBI, prec) == cg.CG_OK
        bd = torch.from_numpy(b).cuda()
        xs = []
        for prec in (cg.CG_PREC_FP64, cg.CG_PREC_FP32_RU):
            xd = torch.zeros_like(bd)
            st, it, rel = cg.cg_solve(h, bd, xd, 1e-9, 5000, cg.CG_PRECOND_JACOBI, prec)
            assert st == cg.CG_OK and rel <= 1e-9
            xs.append((it, xd.cpu().numpy()))
        out.append(xs)
        cg.cg_destroy(h)
    for (i0, x0), (i1, x1) in zip(*out):
        assert i0 == i1 and np.array_equal(x0, x1)


def test_prepare_and_loop_spmv_reject_bad_arguments():
    A = gen.lap2d(10)
    A.vals[A.rowptr[3]:A.rowptr[4]][A.colind[A.rowptr[3]:A.rowptr[4]] == 3] = 0.0  # no Jacobi
    h = cg.cg_create(A.n, *to_device(A))
    assert cg.cg_prepare(h, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP64) == cg.CG_ERR_INVALID
    assert cg.cg_prepare(h, 7, cg.CG_PREC_FP64) == cg.CG_ERR_INVALID
    assert cg.cg_prepare(h, cg.CG_PRECOND_NONE, 9) == cg.CG_ERR_INVALID
    p = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, _ = cg.cg_loop_spmv(h, p, p, cg.CG_PRECOND_NONE, cg.CG_PREC_FP64)
    assert st == cg.CG_ERR_INVALID                       # aliased
    q = torch.zeros_like(p)
    st, _ = cg.cg_loop_spmv(h, p, q, cg.CG_PRECOND_NONE, cg.CG_PREC_FP64, reps=0)
    assert st == cg.CG_ERR_INVALID
    cg.cg_destroy(h)
