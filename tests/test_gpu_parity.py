"""GPU parity: the CUDA path (through the C ABI) against the fp64 oracle on the same
seeded inputs.

Tolerances (derived from the arithmetic, stated here once):
* SpMV: |y_gpu - y_oracle|_i <= 1e-12 * (|A| |x|)_i.  cg_spmv sums each row in the
  oracle's storage order but with fused multiply-adds (one rounding per term where the
  oracle rounds the product and the sum), long rows in a fixed tree; a row of k terms
  then differs by at most about 2k ulp of (|A| |x|)_i, far inside the bound.
* CG: same status; |iters_gpu - iters_oracle| <= max(3, 2% of iters_oracle) (reduction
  order differs, Sec. 3.1 notes the effect); true relative residual of the GPU x,
  recomputed by the oracle in fp64, <= tol; ||x_gpu - x_oracle|| / ||x_oracle|| <=
  2 kappa tol where kappa is known, else 1e-4.
"""
import math

import numpy as np
import pytest

import cgproblems as gen
import oracle
from helpers import adversarial, hub_graph_spd, random_graph_spd, spd_from_pattern, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402


def iters_band(k):
    return max(3, math.ceil(0.02 * k))


def check_spmv(A, seed=1):
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    x = gen.xstar(A.n, seed)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, float("nan"))
    assert cg.cg_spmv(h, xd, yd) == cg.CG_OK
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    ref = oracle.spmv(A, x)
    scale = np.abs(A.to_scipy()) @ np.abs(x)
    err = np.abs(y - ref)
    assert np.all(err <= 1e-12 * scale + 1e-300), f"max rel err {np.max(err / (scale + 1e-300))}"
    cg.cg_destroy(h)
    return y, ref


# ---------------------------------------------------------------- a1: SpMV

@pytest.mark.parametrize("A", [
    gen.lap2d(64),                         # the 64 x 64 Poisson workload: 16 row blocks
    gen.lap2d(37, 9, 0.01),                # ragged tail block
    gen.lap3d7(23),                        # 12167 rows, ragged
    gen.diff3d27(14, 1.0, 3),              # 27-point, 75-row blocks
    gen.q1aniso(45, 1.5, 0.3, 0.05, 2),
], ids=lambda A: A.name)
def test_spmv_matches_oracle(A):
    y, ref = check_spmv(A)
    # same storage order, one rounding less per term: the two agree to a few ulp
    scale = np.abs(A.to_scipy()) @ np.abs(gen.xstar(A.n, 1))
    assert np.max(np.abs(y - ref) / (scale + 1e-300)) <= 64 * 2.0 ** -52


def test_spmv_unaligned_arrays_take_the_scalar_loads():
    """colind and vals that do not start on a 16-byte boundary (views one element into
    larger buffers) must give the same y as aligned copies: the 16-byte loads are used
    only when both arrays allow them."""
    A = gen.lap3d7(23)
    rp, ci, va = to_device(A)
    ci_big = torch.empty(A.nnz + 1, dtype=torch.int32, device="cuda")
    va_big = torch.empty(A.nnz + 1, dtype=torch.float64, device="cuda")
    ci_big[1:].copy_(ci)
    va_big[1:].copy_(va)
    h1 = cg.cg_create(A.n, rp, ci, va)
    h2 = cg.cg_create(A.n, rp, ci_big[1:], va_big[1:])
    x = torch.from_numpy(gen.xstar(A.n, 5)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    assert cg.cg_spmv(h1, x, y1) == cg.CG_OK and cg.cg_spmv(h2, x, y2) == cg.CG_OK
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    cg.cg_destroy(h1)
    cg.cg_destroy(h2)


@pytest.mark.parametrize("case", ["empty_rows", "long_rows", "cap_boundary", "huge_row", "tiny"])
def test_spmv_adversarial_row_lengths(case):
    if case == "empty_rows":
        A = adversarial(3000, 1, empty_every=3)
    elif case == "long_rows":   # rows longer than a row block's 2044 nonzeros
        A = adversarial(6000, 2, long_rows=[(0, 2049), (17, 5000), (5999, 2500)])
    elif case == "cap_boundary":  # around the row-block cap (2044) and the staging size (2048)
        A = adversarial(9000, 6, long_rows=[(0, 2044), (1, 2045), (100, 2047), (5000, 2048),
                                            (8998, 2043), (8999, 2046)])
    elif case == "huge_row":    # one row touching every column
        A = adversarial(20000, 3, long_rows=[(12345, 20000)])
    else:
        A = adversarial(1, 4, max_len=1)
    check_spmv(A)


def test_spmv_all_empty_rows():
    n = 1000
    A = gen.CSR(n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")
    y, _ = check_spmv(A)
    assert np.all(y == 0)


# ---------------------------------------------------------------- a1-a5: solves

def gpu_solve(A, b, tol, maxit, precond, precision=cg.CG_PREC_FP64, x0=None, h=None):
    rp, ci, va = to_device(A)
    own = h is None
    if own:
        h = cg.cg_create(A.n, rp, ci, va)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    st, it, rel = cg.cg_solve(h, bd, xd, tol, maxit, precond, precision)
    info = cg.cg_get_solve_info(h)
    x = xd.cpu().numpy()
    if own:
        cg.cg_destroy(h)
    return st, it, rel, x, info


def compare_solve(A, b, tol, maxit, precond, kappa=None):
    ref = oracle.pcg(A, b, tol=tol, maxit=maxit, precond=precond)
    st, it, rel, x, info = gpu_solve(A, b, tol, maxit, precond)
    assert st == ref.status, (st, ref.status, cg.cg_last_error())
    assert abs(it - ref.iters) <= iters_band(ref.iters), (it, ref.iters)
    rel_or = oracle.true_relres(A, b, x)
    if st == cg.CG_OK:
        assert rel_or <= tol * (1 + 1e-6)
    assert abs(rel - rel_or) <= 1e-6 * rel_or + 1e-15
    xerr = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    bound = 2 * kappa * tol if kappa else 1e-4
    assert xerr <= bound, (xerr, bound)
    return it, ref.iters, xerr, info


def test_cg_poisson_64x64_unpreconditioned():
    """The 64 x 64 Poisson workload: plain CG (Alg. 1), tol 1e-8, maxit 1000."""
    A = gen.lap2d(64)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    kappa = 1.0 / math.tan(math.pi / 130) ** 2
    it, it_or, xerr, _ = compare_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, kappa)
    assert it <= 473  # Chebyshev bound


@pytest.mark.parametrize("N", [20, 33])
def test_jacobi_pcg_poisson_3d(N):
    A = gen.lap3d7(N)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    kappa = 1.0 / math.tan(math.pi / (2 * (N + 1))) ** 2
    compare_solve(A, b, 1e-8, 5000, cg.CG_PRECOND_JACOBI, kappa)


def test_jacobi_pcg_variable_coefficient_27pt():
    A = gen.diff3d27(16, 1.0, 5)
    b = oracle.spmv(A, gen.xstar(A.n, 5))
    compare_solve(A, b, 1e-10, 5000, cg.CG_PRECOND_JACOBI)


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobi_pcg_uneven_rows(seed):
    A = spd_from_pattern(5000, seed, long_rows=[(10, 3000), (4000, 2100), (2500, 2046)])
    b = oracle.spmv(A, gen.xstar(A.n, seed))
    compare_solve(A, b, 1e-9, 2000, cg.CG_PRECOND_JACOBI)


def test_anisotropic_batch_member():
    A = gen.lap2d(70, 9, 2e-3)
    b = oracle.spmv(A, gen.xstar(A.n, 9))
    compare_solve(A, b, 1e-8, 5000, cg.CG_PRECOND_JACOBI)


def test_solve_is_deterministic():
    A = gen.lap3d7(24)
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    r1 = gpu_solve(A, b, 1e-8, 2000, cg.CG_PRECOND_JACOBI)
    r2 = gpu_solve(A, b, 1e-8, 2000, cg.CG_PRECOND_JACOBI)
    assert r1[1] == r2[1] and np.array_equal(r1[3], r2[3])


def test_grid_size_does_not_change_the_answer_beyond_rounding():
    A = gen.lap3d7(24)
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    outs = []
    for g in (1, 3, 0):
        assert cg.cg_set_option(h, cg.CG_OPT_GRID_CTAS, g) == cg.CG_OK
        st, it, rel, x, info = gpu_solve(A, b, 1e-8, 2000, cg.CG_PRECOND_JACOBI, h=h)
        assert st == cg.CG_OK and rel <= 1e-8
        outs.append((it, x, info["grid_ctas"]))
    assert outs[0][2] == 1 and outs[1][2] == 3
    for it, x, _ in outs[1:]:
        assert abs(it - outs[0][0]) <= 3
        assert np.linalg.norm(x - outs[0][1]) <= 1e-5 * np.linalg.norm(outs[0][1])
    cg.cg_destroy(h)


# ---------------------------------------------------------------- mixed precision

@pytest.mark.parametrize("mode", [1, 2], ids=["persistent", "graph"])
@pytest.mark.parametrize("tol_in", [1e-3, 1e-4])
def test_fp32_refinement_reaches_fp64_tolerance(tol_in, mode):
    A = gen.diff3d27(14, 1.0, 7)
    b = oracle.spmv(A, gen.xstar(A.n, 7))
    ref = oracle.pcg_ir(A, b, tol=1e-10, tol_in=tol_in)
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
    assert cg.cg_set_option(h, cg.CG_OPT_IR_TOL_INNER, tol_in) == cg.CG_OK
    st, it, rel, x, info = gpu_solve(A, b, 1e-10, 100000, cg.CG_PRECOND_JACOBI,
                                     cg.CG_PREC_FP32_IR, h=h)
    cg.cg_destroy(h)
    assert st == cg.CG_OK == ref.status
    assert oracle.true_relres(A, b, x) <= 1e-10 * (1 + 1e-6)
    assert abs(info["restarts"] - ref.restarts) <= 1
    assert abs(it - ref.iters) <= max(5, math.ceil(0.1 * ref.iters)), (it, ref.iters)
    fp64 = oracle.pcg(A, b, tol=1e-12, maxit=5000)
    assert np.linalg.norm(x - fp64.x) / np.linalg.norm(fp64.x) <= 1e-7


# ---------------------------------------------------------------- edge cases

def test_zero_rhs():
    A = gen.lap2d(16)
    st, it, rel, x, _ = gpu_solve(A, np.zeros(A.n), 1e-8, 100, cg.CG_PRECOND_JACOBI,
                                  x0=np.ones(A.n))
    assert st == cg.CG_OK and it == 0 and rel == 0.0 and np.all(x == 0)


def test_exact_initial_guess():
    A = gen.lap2d(16)
    xs = gen.xstar(A.n, 3)
    b = oracle.spmv(A, xs)
    st, it, rel, x, _ = gpu_solve(A, b, 1e-8, 100, cg.CG_PRECOND_JACOBI, x0=xs)
    assert st == cg.CG_OK and it == 0


def test_maxit_not_converged_matches_oracle():
    A = gen.lap2d(40)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    ref = oracle.pcg(A, b, tol=1e-12, maxit=25, precond=0)
    st, it, rel, x, _ = gpu_solve(A, b, 1e-12, 25, cg.CG_PRECOND_NONE)
    assert st == cg.CG_NOT_CONVERGED == ref.status and it == 25
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)


def test_maxit_zero():
    A = gen.lap2d(8)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    st, it, rel, x, _ = gpu_solve(A, b, 1e-8, 0, cg.CG_PRECOND_JACOBI)
    assert st == cg.CG_NOT_CONVERGED and it == 0 and np.all(x == 0)


def test_empty_matrix():
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    h = cg.cg_create(0, rp, None, None)
    st, it, rel = cg.cg_solve(h, None, None, 1e-8, 10, 0, 0)
    assert st == cg.CG_OK and it == 0
    cg.cg_destroy(h)


def test_indefinite_matrix_breaks_down():
    import scipy.sparse as sp
    M = sp.diags([1.0, 2.0, -3.0, 4.0] * 50).tocsr()
    A = gen.CSR(200, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data, "indef")
    b = np.ones(200)
    ref = oracle.pcg(A, b, tol=1e-10, maxit=50, precond=0)
    st, *_ = gpu_solve(A, b, 1e-10, 50, cg.CG_PRECOND_NONE)
    assert st == cg.CG_ERR_BREAKDOWN == ref.status


def test_nan_rhs_is_numeric_error():
    A = gen.lap2d(12)
    b = np.ones(A.n)
    b[7] = np.nan
    st, *_ = gpu_solve(A, b, 1e-8, 50, cg.CG_PRECOND_JACOBI)
    assert st == cg.CG_ERR_NUMERIC == oracle.pcg(A, b, tol=1e-8, maxit=50).status


def test_invalid_column_index_rejected():
    A = gen.lap2d(10)
    ci = A.colind.copy()
    ci[37] = A.n  # out of range
    rp, _, va = to_device(A)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.n, rp, torch.from_numpy(ci).cuda(), va)
    assert e.value.status == cg.CG_ERR_INVALID


def test_decreasing_rowptr_rejected():
    A = gen.lap2d(10)
    rp = A.rowptr.copy()
    rp[5], rp[6] = rp[6], rp[5]
    _, ci, va = to_device(A)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.n, torch.from_numpy(rp).cuda(), ci, va)
    assert e.value.status == cg.CG_ERR_INVALID


def test_jacobi_needs_positive_diagonal():
    import scipy.sparse as sp
    M = sp.csr_matrix((np.array([2.0, 3.0]), np.array([0, 2], np.int32),
                       np.array([0, 1, 1, 2], np.int32)), shape=(3, 3))
    A = gen.CSR(3, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data, "nodiag")
    st, *_ = gpu_solve(A, np.ones(3), 1e-8, 10, cg.CG_PRECOND_JACOBI)
    assert st == cg.CG_ERR_INVALID


def test_barrier_timeout_is_reported_and_context_survives():
    """Fault injection on the host's request: CTA 0 skips its arrival at the second grid
    barrier, so every CTA's bounded wait runs out; the solve returns CG_ERR_TIMEOUT and
    the next solve on the same handle works."""
    A = gen.lap2d(64)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_get_matrix_info(h)["grid_ctas"] > 1
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, 1) == cg.CG_OK   # the grid-barrier form
    assert cg.cg_set_option(h, cg.CG_OPT_BARRIER_TIMEOUT_MS, 100) == cg.CG_OK
    assert cg.cg_set_option(h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 2) == cg.CG_OK
    st, *_ = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, h=h)
    assert st == cg.CG_ERR_TIMEOUT
    assert "timed out" in cg.cg_last_error(h)
    assert cg.cg_set_option(h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 0) == cg.CG_OK
    st, it, rel, x, _ = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, h=h)
    assert st == cg.CG_OK and rel <= 1e-8
    cg.cg_destroy(h)


def test_host_buffer_entry_point_matches_device_entry_point():
    A = gen.lap3d7(16)
    b = oracle.spmv(A, gen.xstar(A.n, 4))
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros(A.n, dtype=torch.float64).pin_memory()
    st, it, rel = cg.cg_solve_host(h, bh, xh, 1e-8, 2000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP64)
    st2, it2, rel2, x2, _ = gpu_solve(A, b, 1e-8, 2000, cg.CG_PRECOND_JACOBI, h=h)
    assert st == st2 == cg.CG_OK and it == it2
    assert np.array_equal(xh.numpy(), x2)
    cg.cg_destroy(h)


@pytest.mark.parametrize("mode", [1, 2], ids=["persistent", "graph"])
def test_fp32_refinement_unpreconditioned(mode):
    A = gen.lap2d(48, 9, 0.05)
    b = oracle.spmv(A, gen.xstar(A.n, 11))
    ref = oracle.pcg_ir(A, b, tol=1e-10, tol_in=1e-4, precond=0)
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
    st, it, rel, x, info = gpu_solve(A, b, 1e-10, 100000, cg.CG_PRECOND_NONE, cg.CG_PREC_FP32_IR,
                                     h=h)
    cg.cg_destroy(h)
    assert st == cg.CG_OK == ref.status
    assert oracle.true_relres(A, b, x) <= 1e-10 * (1 + 1e-6)
    assert abs(info["restarts"] - ref.restarts) <= 1
    assert abs(it - ref.iters) <= max(5, math.ceil(0.1 * ref.iters)), (it, ref.iters)


def test_phase_timers_report_time_per_phase():
    A = gen.lap3d7(32)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_PHASE_TIMERS, 1) == cg.CG_OK
    st, it, rel, x, info = gpu_solve(A, b, 1e-8, 2000, cg.CG_PRECOND_JACOBI, h=h)
    cg.cg_destroy(h)
    assert st == cg.CG_OK
    ph = info["phase_ms"]
    assert all(t >= 0 for t in ph) and ph[0] > 0 and ph[2] > 0
    assert sum(ph) <= info["kernel_ms"] * 1.01
    assert info["kernel_bytes_per_iter"] > 0


# ---------------------------------------------------------------- loop forms

def solve_mode(A, b, tol, maxit, precond, mode, x0=None, max_restarts=None):
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
    if max_restarts is not None:
        assert cg.cg_set_option(h, cg.CG_OPT_MAX_RESTARTS, max_restarts) == cg.CG_OK
    out = gpu_solve(A, b, tol, maxit, precond, x0=x0, h=h)
    cg.cg_destroy(h)
    return out


GRAPH_CASES = [
    ("lap2d64_none", lambda: gen.lap2d(64), 0, 1e-8, 1000),
    ("lap3d7_20_jac", lambda: gen.lap3d7(20), 1, 1e-8, 2000),
    ("diff27_12_jac", lambda: gen.diff3d27(12, 1.0, 4), 1, 1e-10, 5000),
    ("uneven_jac", lambda: spd_from_pattern(4000, 3, long_rows=[(5, 2500), (100, 300)]), 1, 1e-9, 3000),
    ("q1_none", lambda: gen.q1aniso(40, 1.5, 0.7, 0.03, 3), 0, 1e-8, 5000),
    ("graph_uniform_jac", lambda: random_graph_spd(6000, 2, 4), 1, 1e-10, 3000),
    ("graph_uniform_none", lambda: random_graph_spd(5000, 5, 3), 0, 1e-10, 3000),
    ("diff27_40_jac", lambda: gen.diff3d27(40, 1.0, 2), 1, 1e-8, 5000),
    # power-law rows: the row-block CSR loop layout (rows sorted by length per block;
    # the graph forms stage its blocks with bulk copies), one with a row past the cap
    ("powerlaw_jac", lambda: gen.graph_spd(20000, 600, 1), 1, 1e-8, 5000),
    ("powerlaw_hub_jac", lambda: hub_graph_spd(20000, 2, 3000), 1, 1e-8, 8000),
]


LOOP_MODES = dict(argvalues=[1, 2, 3, 4], ids=["persistent", "graph", "unrolled", "cluster"])


@pytest.mark.parametrize("name,make,precond,tol,maxit", GRAPH_CASES, ids=[c[0] for c in GRAPH_CASES])
@pytest.mark.parametrize("mode", **LOOP_MODES)
def test_loop_forms_match_oracle(name, make, precond, tol, maxit, mode):
    A = make()
    if mode == 4 and A.n > 32768:
        pytest.skip("the cluster form holds at most 32768 rows")
    b = oracle.spmv(A, gen.xstar(A.n, 6))
    ref = oracle.pcg(A, b, tol=tol, maxit=maxit, precond=precond)
    st, it, rel, x, info = solve_mode(A, b, tol, maxit, precond, mode)
    assert st == ref.status == cg.CG_OK, cg.cg_last_error()
    assert abs(it - ref.iters) <= iters_band(ref.iters), (it, ref.iters)
    rel_or = oracle.true_relres(A, b, x)
    assert rel_or <= tol * (1 + 1e-6)
    assert abs(rel - rel_or) <= 1e-6 * rel_or + 1e-15
    assert np.linalg.norm(x - ref.x) <= 1e-4 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("mode", **LOOP_MODES)
def test_loop_form_edge_cases(mode):
    A = gen.lap2d(24)
    xs = gen.xstar(A.n, 3)
    b = oracle.spmv(A, xs)
    st, it, rel, x, _ = solve_mode(A, np.zeros(A.n), 1e-8, 100, 1, mode, x0=np.ones(A.n))
    assert st == cg.CG_OK and it == 0 and rel == 0.0 and np.all(x == 0)
    st, it, rel, x, _ = solve_mode(A, b, 1e-8, 100, 1, mode, x0=xs)
    assert st == cg.CG_OK and it == 0 and np.array_equal(x, xs)
    ref = oracle.pcg(A, b, tol=1e-12, maxit=20, precond=0)
    st, it, rel, x, _ = solve_mode(A, b, 1e-12, 20, 0, mode)
    assert st == cg.CG_NOT_CONVERGED and it == 20
    assert np.linalg.norm(x - ref.x) <= 1e-10 * np.linalg.norm(ref.x)
    st, it, rel, x, _ = solve_mode(A, b, 1e-8, 0, 1, mode)
    assert st == cg.CG_NOT_CONVERGED and it == 0 and np.all(x == 0)
    import scipy.sparse as sp
    M = sp.diags([1.0, 2.0, -3.0, 4.0] * 50).tocsr()
    Ai = gen.CSR(200, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data, "indef")
    st, *_ = solve_mode(Ai, np.ones(200), 1e-10, 50, 0, mode)
    assert st == cg.CG_ERR_BREAKDOWN
    bn = b.copy()
    bn[7] = np.nan
    st, *_ = solve_mode(A, bn, 1e-8, 50, 1, mode)
    assert st == cg.CG_ERR_NUMERIC


@pytest.mark.parametrize("mode", **LOOP_MODES)
def test_residual_replacement_restarts_match_oracle(mode):
    """A tolerance below what fp64 can attain: the recursive residual passes while the
    true residual stagnates, so the solve restarts from x (reading R3) until the restarts
    run out; the oracle takes the same path."""
    A = gen.diff3d27(10, 1.0, 8)
    b = oracle.spmv(A, gen.xstar(A.n, 8))
    tol, maxit = 1e-17, 3000
    ref = oracle.pcg(A, b, tol=tol, maxit=maxit, precond=1, max_restarts=2)
    st, it, rel, x, info = solve_mode(A, b, tol, maxit, 1, mode, max_restarts=2)
    assert st == ref.status == cg.CG_NOT_CONVERGED
    assert info["restarts"] == ref.restarts
    assert rel <= 1e-12


@pytest.mark.parametrize("mode", [1, 2], ids=["persistent", "graph"])
def test_fp32_refinement_edge_cases(mode):
    A = spd_from_pattern(3000, 4, long_rows=[(7, 2200)])   # variable diagonal, long row
    b = oracle.spmv(A, gen.xstar(A.n, 4))

    def run(bb, maxit, tol=1e-10, x0=None):
        rp, ci, va = to_device(A)
        h = cg.cg_create(A.n, rp, ci, va)
        assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
        out = gpu_solve(A, bb, tol, maxit, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_IR, x0=x0, h=h)
        cg.cg_destroy(h)
        return out

    st, it, rel, x, info = run(np.zeros(A.n), 1000, x0=np.ones(A.n))
    assert st == cg.CG_OK and it == 0 and np.all(x == 0)
    ref = oracle.pcg_ir(A, b, tol=1e-10, tol_in=1e-4)
    st, it, rel, x, info = run(b, 100000)
    assert st == cg.CG_OK == ref.status
    assert oracle.true_relres(A, b, x) <= 1e-10 * (1 + 1e-6)
    assert abs(it - ref.iters) <= max(5, math.ceil(0.1 * ref.iters)), (it, ref.iters)
    st, it, rel, x, info = run(b, 3)                        # inner budget of 3 iterations
    assert st == cg.CG_NOT_CONVERGED and it == 3
    assert abs(rel - oracle.true_relres(A, b, x)) <= 1e-6 * rel


RU_CASES = [("q1_48", lambda: gen.q1aniso(48, 1.5, 0.7, 0.01, 3)),
            ("lap9_50", lambda: gen.lap2d(50, 9, 1e-3)),
            ("diff27_14", lambda: gen.diff3d27(14, 1.0, 2))]


@pytest.mark.parametrize("precond", [cg.CG_PRECOND_JACOBI, cg.CG_PRECOND_NONE], ids=["jacobi", "none"])
@pytest.mark.parametrize("name,make", RU_CASES, ids=[c[0] for c in RU_CASES])
def test_reliable_updates_match_oracle(name, make, precond):
    """fp32 PCG with fp64 reliable updates (R8, default update threshold 0.1) against the
    oracle; it must also need fewer inner iterations than the restarting refinement."""
    A = make()
    b = oracle.spmv(A, gen.xstar(A.n, 4))
    tol = 1e-9
    ref = oracle.pcg_ru(A, b, tol=tol, tol_in=0.1, maxit=100000, precond=precond)
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, rel = cg.cg_solve(h, bd, x, tol, 100000, precond, cg.CG_PREC_FP32_RU)
    info = cg.cg_get_solve_info(h)
    assert st == ref.status == cg.CG_OK, (st, cg.cg_last_error(h))
    # update decisions are taken on fp32 recursive residuals whose rounding differs
    # (Kahan-compensated fp32 sums here, fp64 sums of fp32 products in the oracle)
    assert abs(it - ref.iters) <= max(5, math.ceil(0.1 * ref.iters)), (it, ref.iters)
    assert abs(info["restarts"] - ref.restarts) <= 2, (info["restarts"], ref.restarts)
    xs = x.cpu().numpy()
    assert oracle.true_relres(A, b, xs) <= tol * (1 + 1e-6)
    x2 = torch.zeros_like(bd)
    st2, it_ir, _ = cg.cg_solve(h, bd, x2, tol, 100000, precond, cg.CG_PREC_FP32_IR)
    assert st2 == cg.CG_OK and it < it_ir


@pytest.mark.parametrize("make", [lambda: gen.lap2d(1), lambda: gen.lap2d(5), lambda: random_graph_spd(1000, 3, 5),
                                  lambda: spd_from_pattern(4097, 3, long_rows=[(4096, 900)])],
                         ids=["n1", "n25", "n1000", "n4097_long_last_row"])
def test_cluster_form_ragged_shapes(make):
    """The cluster form's row split (power-of-two rows per CTA, a ragged last CTA, a single
    CTA, one row) against the oracle, Jacobi and plain CG."""
    A = make()
    b = oracle.spmv(A, gen.xstar(A.n, 9))
    for precond in (0, 1):
        ref = oracle.pcg(A, b, tol=1e-10, maxit=3000, precond=precond)
        st, it, rel, x, info = solve_mode(A, b, 1e-10, 3000, precond, 4)
        assert st == ref.status == cg.CG_OK and info["loop_form"] == 4
        assert abs(it - ref.iters) <= iters_band(ref.iters), (it, ref.iters)
        assert oracle.true_relres(A, b, x) <= 1e-10 * (1 + 1e-6)
        assert np.linalg.norm(x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("make,in_smem", [(lambda: gen.lap3d7(24), True),
                                          (lambda: gen.diff3d27(32, 1.0, 5), False)],
                         ids=["lap3d7_24_smem", "diff27_32_global"])
def test_cluster_form_csr_placement(make, in_smem):
    """Each CTA holds its rows of the CSR in shared memory when they fit beside its
    vectors (no bytes from outside the SMs per iteration), else reads them from global
    memory; both against the oracle, and a rerun gives the same bits."""
    A = make()
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    ref = oracle.pcg(A, b, tol=1e-9, maxit=3000, precond=1)
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, 4) == cg.CG_OK
    st, it, rel, x, info = gpu_solve(A, b, 1e-9, 3000, cg.CG_PRECOND_JACOBI, h=h)
    assert st == ref.status == cg.CG_OK and info["loop_form"] == 4
    assert (info["kernel_bytes_per_iter"] == 0) == in_smem
    assert abs(it - ref.iters) <= iters_band(ref.iters), (it, ref.iters)
    assert oracle.true_relres(A, b, x) <= 1e-9 * (1 + 1e-6)
    assert np.linalg.norm(x - ref.x) <= 1e-6 * np.linalg.norm(ref.x)
    st2, it2, rel2, x2, _ = gpu_solve(A, b, 1e-9, 3000, cg.CG_PRECOND_JACOBI, h=h)
    assert st2 == st and it2 == it and rel2 == rel and np.array_equal(x2, x)
    cg.cg_destroy(h)


def test_cluster_form_exchange_timeout_is_reported_and_context_survives():
    """Fault injection on the host's request: CTA 0 of the cluster does not push its
    partial sum of the second exchange (the first p.q), so every CTA's bounded wait runs
    out; the solve returns CG_ERR_TIMEOUT and the next solve on the handle works."""
    A = gen.lap2d(64)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    rp, ci, va = to_device(A)
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, 4) == cg.CG_OK
    assert cg.cg_set_option(h, cg.CG_OPT_BARRIER_TIMEOUT_MS, 100) == cg.CG_OK
    assert cg.cg_set_option(h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 2) == cg.CG_OK
    st, *_, info = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, h=h)
    assert st == cg.CG_ERR_TIMEOUT and info["loop_form"] == 4
    assert "timed out" in cg.cg_last_error(h)
    assert cg.cg_set_option(h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 0) == cg.CG_OK
    st, it, rel, x, info = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, h=h)
    assert st == cg.CG_OK and rel <= 1e-8 and info["loop_form"] == 4
    cg.cg_destroy(h)


def test_cluster_form_is_chosen_for_small_systems_and_refuses_large_ones():
    """Automatic loop form: the 64 x 64 Poisson system (4096 rows) runs in one thread-block
    cluster; forcing the cluster form beyond its 32768 rows is refused."""
    A = gen.lap2d(64)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    st, it, rel, x, info = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE)
    assert st == cg.CG_OK and info["loop_form"] == 4 and info["kernel_launches"] == 1
    ref = oracle.pcg(A, b, tol=1e-8, maxit=1000, precond=0)
    assert abs(it - ref.iters) <= iters_band(ref.iters)
    rp, ci, va = to_device(A)                # a grid size given: the persistent form
    h = cg.cg_create(A.n, rp, ci, va)
    assert cg.cg_set_option(h, cg.CG_OPT_GRID_CTAS, 5) == cg.CG_OK
    st, it2, _, _, info = gpu_solve(A, b, 1e-8, 1000, cg.CG_PRECOND_NONE, h=h)
    assert st == cg.CG_OK and info["loop_form"] == 1 and info["grid_ctas"] == 5
    assert abs(it2 - ref.iters) <= iters_band(ref.iters)
    cg.cg_destroy(h)
    B = gen.lap3d7(33)                       # 35937 rows
    st, *_ = solve_mode(B, oracle.spmv(B, gen.xstar(B.n, 1)), 1e-8, 100, 1, 4)
    assert st == cg.CG_ERR_INVALID
