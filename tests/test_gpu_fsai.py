"""GPU parity of the FSAI preconditioner (cg_fsai_classic / cg_fsai_set_factor and
cg_solve with CG_PRECOND_FSAI) against the oracle (oracle/fsai.py, oracle.c R7).

Tolerances: classic factor values to 1e-10 relative (a Cholesky solve against the
oracle's LU solve of the same 2..16-row systems); solves as for cg_solve: same status,
|iters - iters_oracle| <= max(3, 2%), true relative residual <= tol, x to the oracle's
x within 1e-4 relative."""
import math

import numpy as np
import pytest

import cgproblems as gen
import oracle
from oracle import fsai
from helpers import to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402


def iters_band(k):
    return max(3, math.ceil(0.02 * k))


def ru_band(k):
    """Reliable updates take their update decisions on fp32 recursive residuals, whose
    rounding differs between the kernels (Kahan-compensated fp32 sums) and the oracle
    (fp64 sums of fp32 products); the update points, and with them the count, shift."""
    return max(5, math.ceil(0.1 * k))


def handle(A):
    return cg.cg_create(A.n, *to_device(A))


CASES = [
    ("q1_24", lambda: gen.q1aniso(24, 1.5, 0.6, 0.01, 3)),
    ("q1_37_ragged", lambda: gen.q1aniso(37, 1.5, 2.4, 0.2, 5)),
    ("lap2d_9pt", lambda: gen.lap2d(30, 9, 1e-2)),
    ("diff27", lambda: gen.diff3d27(9, 1.0, 1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_classic_factor_matches_oracle(name, make):
    A = make()
    h = handle(A)
    assert cg.cg_fsai_classic(h) == cg.CG_OK, cg.cg_last_error(h)
    st, g, kind = cg.cg_fsai_get_factor(h)
    assert st == cg.CG_OK and kind == 1
    ref = fsai.classic(A)
    g = g.cpu().numpy()
    assert np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-300)) <= 1e-10


@pytest.mark.parametrize("precision", [cg.CG_PREC_FP64, cg.CG_PREC_FP32_IR, cg.CG_PREC_FP32_RU],
                         ids=["fp64", "fp32_ir", "fp32_ru"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fsai_pcg_matches_oracle(name, make, precision):
    A = make()
    g = fsai.classic(A)
    b = oracle.spmv(A, gen.xstar(A.n, 7))
    tol = 1e-9
    h = handle(A)
    assert cg.cg_fsai_set_factor(h, torch.from_numpy(g).cuda()) == cg.CG_OK
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, tol, 20000, cg.CG_PRECOND_FSAI, precision)
    info = cg.cg_get_solve_info(h)
    assert info["precond_used"] == cg.CG_PRECOND_FSAI
    if precision == cg.CG_PREC_FP64:
        ref = fsai.pcg(A, g, b, tol=tol, maxit=20000)
    elif precision == cg.CG_PREC_FP32_IR:
        ref = fsai.pcg_ir(A, g, b, tol=tol, tol_in=1e-4, maxit=20000)
    else:
        ref = fsai.pcg_ir(A, g, b, tol=tol, tol_in=0.1, maxit=20000, carry=True)
    assert st == ref.status == cg.CG_OK, (st, ref.status, cg.cg_last_error(h))
    band = iters_band(ref.iters) if precision != cg.CG_PREC_FP32_RU else ru_band(ref.iters)
    assert abs(it - ref.iters) <= band, (it, ref.iters)
    xs = x.cpu().numpy()
    rel_or = oracle.true_relres(A, b, xs)
    assert rel_or <= tol * (1 + 1e-6)
    assert abs(rel - rel_or) <= 1e-6 * rel_or + 1e-15
    assert np.linalg.norm(xs - ref.x) <= 1e-4 * np.linalg.norm(ref.x)
    # the GPU's own classic factor gives the same solve
    h2 = handle(A)
    assert cg.cg_fsai_classic(h2) == cg.CG_OK
    x2 = torch.zeros_like(bd)
    st2, it2, _ = cg.cg_solve(h2, bd, x2, tol, 20000, cg.CG_PRECOND_FSAI, precision)
    assert st2 == cg.CG_OK and abs(it2 - it) <= 1


def test_fsai_beats_jacobi_on_anisotropic_q1():
    A = gen.q1aniso(64, 1.5, 0.3, 1e-2, 11)
    b = oracle.spmv(A, gen.xstar(A.n, 3))
    h = handle(A)
    assert cg.cg_fsai_classic(h) == cg.CG_OK
    bd = torch.from_numpy(b).cuda()
    its = {}
    for pc in (cg.CG_PRECOND_JACOBI, cg.CG_PRECOND_FSAI):
        x = torch.zeros_like(bd)
        st, it, rel = cg.cg_solve(h, bd, x, 1e-8, 20000, pc)
        assert st == cg.CG_OK and rel <= 1e-8
        its[pc] = it
    ref_j = oracle.pcg(A, b, tol=1e-8, maxit=20000, precond=1)
    ref_f = fsai.pcg(A, fsai.classic(A), b, tol=1e-8, maxit=20000)
    assert abs(its[cg.CG_PRECOND_JACOBI] - ref_j.iters) <= iters_band(ref_j.iters)
    assert abs(its[cg.CG_PRECOND_FSAI] - ref_f.iters) <= iters_band(ref_f.iters)
    assert its[cg.CG_PRECOND_FSAI] < 0.7 * its[cg.CG_PRECOND_JACOBI]


def test_jacobi_factor_reproduces_jacobi():
    """G = D^-1/2 set by the caller: G^T G = D^-1, so the counts equal Jacobi-PCG's."""
    A = gen.q1aniso(40, 1.5, 1.0, 0.05, 2)
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    gj = np.where(rows == tci, 1.0 / np.sqrt(fsai.diag(A))[rows], 0.0)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    h = handle(A)
    assert cg.cg_fsai_set_factor(h, torch.from_numpy(gj).cuda()) == cg.CG_OK
    assert cg.cg_fsai_get_factor(h)[2] == 3
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, _ = cg.cg_solve(h, bd, x, 1e-9, 5000, cg.CG_PRECOND_FSAI)
    ref = oracle.pcg(A, b, tol=1e-9, maxit=5000, precond=1)
    assert st == cg.CG_OK and abs(it - ref.iters) <= iters_band(ref.iters)


def test_fsai_without_a_factor_falls_back_to_jacobi():
    A = gen.q1aniso(20, 1.5, 0.5, 0.1, 4)
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    h = handle(A)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, 1e-8, 5000, cg.CG_PRECOND_FSAI)
    assert st == cg.CG_OK and rel <= 1e-8
    assert cg.cg_get_solve_info(h)["precond_used"] == cg.CG_PRECOND_JACOBI
    ref = oracle.pcg(A, b, tol=1e-8, maxit=5000, precond=1)
    assert abs(it - ref.iters) <= iters_band(ref.iters)


def test_fsai_edge_cases():
    A = gen.q1aniso(16, 1.5, 0.5, 0.1, 6)
    h = handle(A)
    assert cg.cg_fsai_classic(h) == cg.CG_OK
    g = fsai.classic(A)
    # b = 0: x = 0, no iterations
    bd = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    x = torch.ones_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, 1e-8, 100, cg.CG_PRECOND_FSAI)
    assert st == cg.CG_OK and it == 0 and torch.all(x == 0)
    # maxit reached: not converged, same count and residual as the oracle
    b = oracle.spmv(A, gen.xstar(A.n, 5))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, 1e-12, 5, cg.CG_PRECOND_FSAI)
    ref = fsai.pcg(A, g, b, tol=1e-12, maxit=5)
    assert st == ref.status == cg.CG_NOT_CONVERGED and it == ref.iters == 5
    assert abs(rel - ref.relres_true) <= 1e-8 * ref.relres_true
    # a factor with a non-positive diagonal is refused
    bad = g.copy()
    trp, tci, _ = fsai.tril(A)
    bad[trp[3 + 1] - 1] = -1.0
    assert cg.cg_fsai_set_factor(h, torch.from_numpy(bad).cuda()) == cg.CG_ERR_INVALID
    assert "diagonal" in cg.cg_last_error(h)


def test_fsai_rejects_unsuitable_matrices():
    # an indefinite matrix: a local matrix is not SPD
    M = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    import scipy.sparse as sp
    S = sp.csr_matrix(M)
    A = gen.CSR(3, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data, "indef")
    h = handle(A)
    assert cg.cg_fsai_classic(h) == cg.CG_ERR_INVALID
    assert "not SPD" in cg.cg_last_error(h)
    # unsorted columns in a row
    A = gen.lap2d(5)
    ci = A.colind.copy()
    ci[[5, 6]] = ci[[6, 5]]
    va = A.vals.copy()
    va[[5, 6]] = va[[6, 5]]
    h = handle(gen.CSR(A.n, A.rowptr, ci, va, "unsorted"))
    assert cg.cg_fsai_classic(h) == cg.CG_ERR_INVALID
    assert "increasing" in cg.cg_last_error(h)


@pytest.mark.parametrize("precision", [cg.CG_PREC_FP32_IR, cg.CG_PREC_FP32_RU], ids=["fp32_ir", "fp32_ru"])
@pytest.mark.parametrize("mode", [1, 2, 3], ids=["persistent", "graph", "unrolled"])
@pytest.mark.parametrize("name,make", CASES[:3] + [("q1_260", lambda: gen.q1aniso(260, 1.5, 1.9, 0.004, 8))],
                         ids=[c[0] for c in CASES[:3]] + ["q1_260"])
def test_fsai_refinement_loop_forms_match_oracle(name, make, mode, precision):
    """The loop forms of the fp32 FSAI refinement (the persistent kernel, the graph of
    phase kernels under WHILE nodes, and the same kernels in unrolled graphs relaunched by
    the host) against the oracle; the automatic choice is the graph form from 2^21 rows."""
    A = make()
    g = fsai.classic(A)
    b = oracle.spmv(A, gen.xstar(A.n, 9))
    tol = 1e-9
    h = handle(A)
    assert cg.cg_fsai_set_factor(h, torch.from_numpy(g).cuda()) == cg.CG_OK
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, tol, 100000, cg.CG_PRECOND_FSAI, precision)
    info = cg.cg_get_solve_info(h)
    assert info["loop_form"] == mode
    carry = precision == cg.CG_PREC_FP32_RU
    ref = fsai.pcg_ir(A, g, b, tol=tol, tol_in=0.1 if carry else 1e-4, maxit=100000, carry=carry)
    assert st == ref.status == cg.CG_OK, (st, cg.cg_last_error(h))
    band = ru_band(ref.iters) if carry else iters_band(ref.iters)
    assert abs(it - ref.iters) <= band, (it, ref.iters)
    assert abs(info["restarts"] - ref.restarts) <= (2 if carry else 0)
    xs = x.cpu().numpy()
    assert oracle.true_relres(A, b, xs) <= tol * (1 + 1e-6)
    assert abs(rel - oracle.true_relres(A, b, xs)) <= 1e-6 * rel + 1e-15
    # auto picks the graph form from 2^21 rows
    h2 = handle(A)
    assert cg.cg_fsai_set_factor(h2, torch.from_numpy(g).cuda()) == cg.CG_OK
    x2 = torch.zeros_like(bd)
    assert cg.cg_solve(h2, bd, x2, tol, 100000, cg.CG_PRECOND_FSAI, precision)[0] == cg.CG_OK
    assert cg.cg_get_solve_info(h2)["loop_form"] == (2 if A.n >= 1 << 21 else 1)


@pytest.mark.parametrize("precision", [cg.CG_PREC_FP32_IR, cg.CG_PREC_FP32_RU], ids=["fp32_ir", "fp32_ru"])
def test_fsai_unrolled_graph_equals_while_graph(precision):
    """The unrolled graphs run the WHILE graph's kernels in the same order with the same
    grids, so the two forms give the same x bit for bit and the same counts."""
    A = gen.q1aniso(130, 1.5, 0.4, 0.01, 12)
    g = fsai.classic(A)
    b = oracle.spmv(A, gen.xstar(A.n, 3))
    bd = torch.from_numpy(b).cuda()
    out = {}
    for mode in (2, 3):
        h = handle(A)
        assert cg.cg_fsai_set_factor(h, torch.from_numpy(g).cuda()) == cg.CG_OK
        assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
        x = torch.zeros_like(bd)
        st, it, rel = cg.cg_solve(h, bd, x, 1e-9, 100000, cg.CG_PRECOND_FSAI, precision)
        assert st == cg.CG_OK, cg.cg_last_error(h)
        info = cg.cg_get_solve_info(h)
        out[mode] = (x.cpu().numpy(), it, info["restarts"], rel)
    assert np.array_equal(out[2][0], out[3][0])
    assert out[2][1:] == out[3][1:]


def with_explicit_zero(A, i, j):
    """A copy of A with an explicit zero stored at (i, j), (i, j) not yet stored."""
    cols = A.colind[A.rowptr[i]:A.rowptr[i + 1]]
    assert j not in cols
    at = A.rowptr[i] + int(np.searchsorted(cols, j))
    rowptr = A.rowptr.copy()
    rowptr[i + 1:] += 1
    colind = np.insert(A.colind, at, j).astype(np.int32)
    vals = np.insert(A.vals, at, 0.0)
    return gen.CSR(A.n, rowptr, colind, vals, A.name + "_unsym")


def test_pattern_of_a_structurally_unsymmetric_matrix():
    """An explicit zero stored below the diagonal without its mirror makes the stored
    structure unsymmetric, so column j of tril(A) is no longer the upper half of row j
    and the pattern is built on the host.  The classic factor (whose pattern includes
    the stored zero) must match the oracle, and the preconditioned solve converge like
    the oracle's."""
    A = with_explicit_zero(gen.lap2d(12), 40, 3)
    h = handle(A)
    assert cg.cg_fsai_classic(h) == cg.CG_OK, cg.cg_last_error(h)
    st, g, kind = cg.cg_fsai_get_factor(h)
    ref = fsai.classic(A)
    assert g.numel() == ref.size == fsai.tril(A)[1].size
    g = g.cpu().numpy()
    assert np.max(np.abs(g - ref) / np.maximum(np.abs(ref), 1e-300)) <= 1e-10
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, 1e-10, 5000, cg.CG_PRECOND_FSAI, cg.CG_PREC_FP64)
    r = fsai.pcg(A, ref, b, tol=1e-10, maxit=5000)
    assert st == cg.CG_OK and abs(it - r.iters) <= iters_band(r.iters)
    assert oracle.true_relres(A, b, x.cpu().numpy()) <= 1e-10 * (1 + 1e-6)
