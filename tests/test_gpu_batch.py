"""GPU parity of the batched solve (cg_solve_batch): every system of a batch must be
what the single-system oracle gives for it.

Tolerances, as for cg_solve: same status per system; |iters - iters_oracle| <=
max(3, 2% of iters_oracle); the true relative residual of each returned x,
recomputed by the oracle in fp64, <= tol and equal to the reported one to 1e-6
relative; ||x - x_oracle|| / ||x_oracle|| <= 1e-4.  The schedule (grid size, graph
or direct launch) must not change the answer at all: each system's sums are
formed over its own (4096-row group, warp) partials in a fixed order, so results
are compared bit for bit.
"""
import math

import numpy as np
import pytest

import cgproblems as gen
import oracle
from helpers import random_graph_spd, spd_from_pattern, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402


def iters_band(k):
    return max(3, math.ceil(0.02 * k))


def mixed_systems():
    """Uneven sizes (1 row to several tiles, ragged tails), 5- and 9-point
    anisotropic Laplacians, a variable diagonal, random row lengths."""
    return [
        gen.lap2d(20, 5, 1.0),
        gen.lap2d(33, 9, 1e-2),
        gen.lap2d(7, 5, 3e-3),
        random_graph_spd(1000, 3, 3),
        gen.diff3d27(9, 1.0, 4),
        spd_from_pattern(700, 5, long_rows=[(3, 300)]),
        gen.CSR(1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5]), "one_row"),
        gen.lap2d(48, 9, 0.3),
        gen.q1aniso(30, 1.5, 0.7, 0.05, 9),
    ]


class Batch:
    def __init__(self, systems):
        self.systems = systems
        self.dev = [to_device(A) for A in systems]
        self.h = cg.cg_batch_create([d[0] for d in self.dev], [d[1] for d in self.dev],
                                    [d[2] for d in self.dev])

    def solve(self, bs, tol, maxit, precond, x0s=None, check=True):
        bd = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
        if x0s is None:
            xd = [torch.zeros_like(b) for b in bd]
        else:
            xd = [torch.from_numpy(np.array(x, dtype=np.float64)).cuda() for x in x0s]
        st, its, rels = cg.cg_solve_batch(self.h, bd, xd, tol, maxit, precond)
        torch.cuda.synchronize()
        per = [cg.cg_batch_get_system(self.h, s) for s in range(len(bs))]
        return st, its, rels, [x.cpu().numpy() for x in xd], per


def rhs(systems, seed=0):
    return [oracle.spmv(A, gen.xstar(A.n, seed + i)) for i, A in enumerate(systems)]


def check_against_oracle(systems, bs, res, tol, maxit, precond, max_restarts=3, xtol=1e-4):
    st, its, rels, xs, per = res
    for s, A in enumerate(systems):
        ref = oracle.pcg(A, bs[s], tol=tol, maxit=maxit, precond=precond, max_restarts=max_restarts)
        assert per[s]["status"] == ref.status, (s, A.name, per[s], ref.status)
        assert per[s]["iters"] == its[s]
        assert abs(its[s] - ref.iters) <= iters_band(ref.iters), (s, A.name, its[s], ref.iters)
        if np.linalg.norm(bs[s]) == 0:
            assert np.all(xs[s] == 0) and its[s] == 0
            continue
        rel_or = oracle.true_relres(A, bs[s], xs[s])
        if ref.status == cg.CG_OK:
            assert rel_or <= tol * (1 + 1e-6), (s, A.name, rel_or)
            xerr = np.linalg.norm(xs[s] - ref.x) / np.linalg.norm(ref.x)
            assert xerr <= xtol, (s, A.name, xerr)
        assert abs(rels[s] - rel_or) <= 1e-6 * rel_or + 1e-15, (s, A.name, rels[s], rel_or)


@pytest.mark.parametrize("precond", [cg.CG_PRECOND_JACOBI, cg.CG_PRECOND_NONE], ids=["jacobi", "none"])
def test_mixed_batch_matches_oracle_per_system(precond):
    systems = mixed_systems()
    bs = rhs(systems)
    B = Batch(systems)
    res = B.solve(bs, 1e-8, 5000, precond)
    assert res[0] == cg.CG_OK, cg.cg_last_error(B.h)
    check_against_oracle(systems, bs, res, 1e-8, 5000, precond)
    info = cg.cg_get_solve_info(B.h)
    assert info["iters"] == max(res[1]) and info["kernel_launches"] == 4
    tune = cg.cg_batch_get_tuning(B.h, precond)
    assert info["grid_ctas"] == tune["grids"][tune["chosen"]]


def test_anisotropic_members_of_the_512_system_family():
    """Members of the 512-system workload family (5-/9-point, eps log-uniform in
    [1e-3, 1]) at sides the oracle finishes quickly."""
    params = gen.batch_members(24, seed=7, side_lo=8, side_hi=72)
    systems = [gen.lap2d(side, pts, eps) for side, pts, eps in params]
    bs = rhs(systems, 100)
    B = Batch(systems)
    res = B.solve(bs, 1e-8, 20000, cg.CG_PRECOND_JACOBI)
    assert res[0] == cg.CG_OK
    check_against_oracle(systems, bs, res, 1e-8, 20000, cg.CG_PRECOND_JACOBI)


def test_schedule_does_not_change_the_answer():
    """Grid size (autotuned and forced) and launch form leave every bit of x unchanged."""
    systems = mixed_systems()
    bs = rhs(systems, 3)
    B = Batch(systems)
    base = B.solve(bs, 1e-9, 5000, cg.CG_PRECOND_JACOBI)
    assert base[0] == cg.CG_OK
    tune = cg.cg_batch_get_tuning(B.h, cg.CG_PRECOND_JACOBI)
    assert len(tune["grids"]) >= 2 and 0 <= tune["chosen"] < len(tune["grids"])
    assert set(tune["ctas_per_sm"]) <= {3, 4, 5}
    assert all(ms > 0 for ms in tune["ms"])
    for grid, mode in ((1, 2), (7, 1), (300, 2), (0, 1)):
        assert cg.cg_set_option(B.h, cg.CG_OPT_GRID_CTAS, grid) == cg.CG_OK
        assert cg.cg_set_option(B.h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
        out = B.solve(bs, 1e-9, 5000, cg.CG_PRECOND_JACOBI)
        assert out[1] == base[1]
        for a, b in zip(out[3], base[3]):
            assert np.array_equal(a, b)
        info = cg.cg_get_solve_info(B.h)
        if grid:
            assert info["grid_ctas"] == grid
        assert info["loop_form"] == mode


def test_autotuner_trials_leave_the_initial_guess_alone():
    systems = mixed_systems()[:5]
    bs = rhs(systems, 11)
    x0s = [gen.xstar(A.n, 50 + i) * 0.5 for i, A in enumerate(systems)]
    B1 = Batch(systems)  # first solve runs the autotuner
    r1 = B1.solve(bs, 1e-8, 5000, cg.CG_PRECOND_JACOBI, x0s)
    r2 = B1.solve(bs, 1e-8, 5000, cg.CG_PRECOND_JACOBI, x0s)  # tuned already
    assert r1[1] == r2[1]
    for a, b in zip(r1[3], r2[3]):
        assert np.array_equal(a, b)
    check_against_oracle(systems, bs, r1, 1e-8, 5000, cg.CG_PRECOND_JACOBI)


def test_per_system_edge_cases():
    """b = 0 (x = 0, no iterations), an exact initial guess, maxit reached for one
    system only, and an indefinite system that breaks down, in one batch: each
    system gets the oracle's status and the others are unaffected."""
    good = gen.lap2d(30, 5, 1.0)
    hard = gen.lap2d(60, 9, 1e-3)
    indef = gen.CSR(3, np.array([0, 1, 2, 3], np.int32), np.array([0, 1, 2], np.int32),
                    np.array([1.0, -1.0, 1.0]), "indefinite_diag")
    systems = [good, gen.lap2d(12), hard, good, indef]
    bs = rhs(systems, 20)
    bs[1] = np.zeros(systems[1].n)
    x0s = [np.zeros(A.n) for A in systems]
    x0s[3] = gen.xstar(good.n, 23)     # bs[3] = A x0s[3]: converged before any SpMV
    bs[4] = np.array([1.0, 1.0, 1.0])
    B = Batch(systems)
    maxit = 40
    res = B.solve(bs, 1e-8, maxit, cg.CG_PRECOND_NONE, x0s)
    st, its, rels, xs, per = res
    assert st == cg.CG_ERR_BREAKDOWN
    assert [p["status"] for p in per] == [cg.CG_NOT_CONVERGED, cg.CG_OK, cg.CG_NOT_CONVERGED, cg.CG_OK,
                                         cg.CG_ERR_BREAKDOWN]
    assert its[1] == 0 and np.all(xs[1] == 0)
    assert its[3] == 0
    for s in (0, 2, 4):
        ref = oracle.pcg(systems[s], bs[s], x0=x0s[s], tol=1e-8, maxit=maxit, precond=0)
        assert per[s]["status"] == ref.status and its[s] == ref.iters
        assert abs(rels[s] - ref.relres_true) <= 1e-9 * ref.relres_true + 1e-15


def test_residual_replacement_restarts_match_oracle():
    """A tolerance below what fp64 reaches: every system uses up its restarts and ends
    not converged, as the oracle does."""
    systems = [gen.lap2d(25, 5, 1.0), gen.lap2d(40, 9, 0.1)]
    bs = rhs(systems, 31)
    B = Batch(systems)
    assert cg.cg_set_option(B.h, cg.CG_OPT_MAX_RESTARTS, 2) == cg.CG_OK
    res = B.solve(bs, 1e-17, 3000, cg.CG_PRECOND_JACOBI)
    for s, A in enumerate(systems):
        ref = oracle.pcg(A, bs[s], tol=1e-17, maxit=3000, precond=1, max_restarts=2)
        assert res[4][s]["status"] == ref.status == cg.CG_NOT_CONVERGED
        assert res[4][s]["restarts"] == ref.restarts


def test_barrier_timeout_is_reported_and_the_handle_survives():
    systems = mixed_systems()[:3]
    bs = rhs(systems, 40)
    B = Batch(systems)
    assert cg.cg_set_option(B.h, cg.CG_OPT_GRID_CTAS, 8) == cg.CG_OK
    assert cg.cg_set_option(B.h, cg.CG_OPT_BARRIER_TIMEOUT_MS, 200) == cg.CG_OK
    assert cg.cg_set_option(B.h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 5) == cg.CG_OK
    res = B.solve(bs, 1e-8, 5000, cg.CG_PRECOND_JACOBI)
    assert res[0] == cg.CG_ERR_TIMEOUT
    assert "timed out" in cg.cg_last_error(B.h)
    assert cg.cg_set_option(B.h, cg.CG_OPT_DEBUG_SKIP_ARRIVAL, 0) == cg.CG_OK
    res = B.solve(bs, 1e-8, 5000, cg.CG_PRECOND_JACOBI)
    assert res[0] == cg.CG_OK
    check_against_oracle(systems, bs, res, 1e-8, 5000, cg.CG_PRECOND_JACOBI)


def test_batch_argument_checks():
    systems = mixed_systems()[:2]
    B = Batch(systems)
    bs = [torch.zeros(A.n, dtype=torch.float64, device="cuda") for A in systems]
    xs = [torch.zeros_like(b) for b in bs]
    lib = cg.load()
    # single-system calls refuse a batch handle
    assert cg.cg_solve(B.h, bs[0], xs[0])[0] == cg.CG_ERR_INVALID
    assert cg.cg_spmv(B.h, bs[0], xs[0]) == cg.CG_ERR_INVALID
    # unknown precision; unknown preconditioner; loop mode 3
    st, _, _ = cg.cg_solve_batch(B.h, bs, xs, 1e-8, 10, cg.CG_PRECOND_JACOBI, 9)
    assert st == cg.CG_ERR_INVALID
    assert cg.cg_solve_batch(B.h, bs, xs, 1e-8, 10, 7)[0] == cg.CG_ERR_INVALID
    assert cg.cg_solve_batch(B.h, bs, xs, -1.0, 10)[0] == cg.CG_ERR_INVALID
    # a batch call on a single-system handle
    A = gen.lap2d(5)
    h1 = cg.cg_create(A.n, *to_device(A))
    assert cg.cg_solve_batch(h1, bs[:1], xs[:1])[0] == cg.CG_ERR_INVALID
    # creation errors name the offending system
    bad = gen.lap2d(6)
    ci = bad.colind.copy()
    ci[5] = 999
    bad = gen.CSR(bad.n, bad.rowptr, ci, bad.vals, "bad_col")
    with pytest.raises(cg.CGError) as e:
        Batch([systems[0], bad])
    assert "system 1" in str(e.value)
    out = __import__("ctypes").c_void_p()
    assert lib.cg_batch_create(0, None, None, None, None, __import__("ctypes").byref(out)) == cg.CG_ERR_INVALID
    with pytest.raises(cg.CGError):
        cg.cg_batch_get_system(B.h, 5)


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden", "batch512_oracle.json")


def test_full_512_system_batch_matches_the_oracle_counts():
    """The 512-system workload at full size, in the benchmark's launch configuration
    (autotuned grid, graph-captured launch): every member converges, its fp64 true
    residual recomputed by the oracle is <= tol, and its iteration count is within
    the band of the oracle's own count (stored by tests/golden/make_batch_iterations.py)."""
    import json
    import os
    if not os.path.exists(GOLDEN):
        pytest.skip("golden batch counts not generated")
    gold = json.load(open(GOLDEN))
    params = gen.batch_members(gold["count"], gold["seed"])
    systems = [gen.lap2d(side, pts, eps) for side, pts, eps in params]
    bs = [oracle.spmv(A, gen.xstar(A.n, i)) for i, A in enumerate(systems)]
    B = Batch(systems)
    st, its, rels, xs, per = B.solve(bs, gold["tol"], gold["maxit"], cg.CG_PRECOND_JACOBI)
    assert st == cg.CG_OK, cg.cg_last_error(B.h)
    assert cg.cg_get_solve_info(B.h)["loop_form"] == 2
    for i, (A, m) in enumerate(zip(systems, gold["members"])):
        assert (m["side"], m["points"]) == params[i][:2]
        assert per[i]["status"] == m["status"] == cg.CG_OK
        assert abs(its[i] - m["iters"]) <= iters_band(m["iters"]), (i, its[i], m["iters"])
        rel_or = oracle.true_relres(A, bs[i], xs[i])
        assert rel_or <= gold["tol"] * (1 + 1e-6), (i, rel_or)
        assert abs(rels[i] - rel_or) <= 1e-6 * rel_or + 1e-15


def test_sudden_convergence_takes_the_exact_stopping_test():
    """Systems whose residual collapses in one iteration (few distinct eigenvalues of the
    scaled matrix): the recursive test must still be taken on the exact r.r, so the
    counts equal the oracle's."""
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    d = rng.uniform(1.0, 10.0, 900)
    diag = sp.diags(d).tocsr()
    blk = sp.block_diag([sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 2.0]]))] * 450).tocsr()
    scale = sp.diags(rng.uniform(0.5, 2.0, 900))
    blk = (scale @ blk @ scale).tocsr()
    mats = []
    for M, name in ((diag, "diag"), (blk, "blocks2x2")):
        M.sort_indices()
        mats.append(gen.CSR(900, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                            M.data.astype(np.float64), name))
    systems = mats + [gen.lap2d(16)]
    bs = rhs(systems, 61)
    B = Batch(systems)
    res = B.solve(bs, 1e-10, 100, cg.CG_PRECOND_JACOBI)
    assert res[0] == cg.CG_OK
    for s, A in enumerate(systems):
        ref = oracle.pcg(A, bs[s], tol=1e-10, maxit=100, precond=1)
        assert res[1][s] == ref.iters, (A.name, res[1][s], ref.iters)
    assert res[1][0] == 1 and res[1][1] == 2
    check_against_oracle(systems, bs, res, 1e-10, 100, cg.CG_PRECOND_JACOBI)


def test_a_breakdown_in_the_diagonal_layout_stays_in_its_system():
    """Stencil members use the diagonal layout, whose gathers are clamped into the
    member's own rows.  An indefinite 5-point member (the Laplacian shifted by -3 I)
    that breaks down between healthy 5- and 9-point members gets the oracle's status,
    and the healthy members' results are bit for bit those of a batch without it."""
    good = [gen.lap2d(24, 5, 1.0), gen.lap2d(31, 9, 0.05), gen.lap2d(17, 5, 0.2)]
    L = gen.lap2d(20, 5, 1.0)
    vals = L.vals.copy()
    rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
    vals[L.colind == rows] -= 3.0
    bad = gen.CSR(L.n, L.rowptr, L.colind, vals, "shifted_lap2d")
    bs_good = rhs(good, 40)
    b_bad = oracle.spmv(bad, gen.xstar(bad.n, 7))
    maxit = 2000
    res_mixed = Batch([good[0], bad, good[1], good[2]]).solve(
        [bs_good[0], b_bad, bs_good[1], bs_good[2]], 1e-9, maxit, cg.CG_PRECOND_NONE)
    res_good = Batch(good).solve(bs_good, 1e-9, maxit, cg.CG_PRECOND_NONE)
    ref_bad = oracle.pcg(bad, b_bad, tol=1e-9, maxit=maxit, precond=0)
    assert ref_bad.status in (cg.CG_ERR_BREAKDOWN, cg.CG_NOT_CONVERGED)
    assert res_mixed[4][1]["status"] == ref_bad.status
    for k, s in enumerate((0, 2, 3)):
        assert res_mixed[4][s]["status"] == cg.CG_OK
        assert res_mixed[1][s] == res_good[1][k]
        assert np.array_equal(res_mixed[3][s], res_good[3][k])
