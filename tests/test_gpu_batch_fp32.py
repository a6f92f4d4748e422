"""GPU parity of the batched solve in fp32 with fp64 refinement: cg_solve_batch with
CG_PREC_FP32_RU (fp32 Jacobi-PCG with fp64 reliable updates, reading R8) and
CG_PREC_FP32_IR (restarting refinement, R6) must give, for every system of a batch,
what the single-system oracle gives for it (oracle.pcg_ru / oracle.pcg_ir).

Tolerances, as for the single-system refinement: same status per system; the inner
iteration count within max(5, 10 %) of the oracle's (update points are decided on fp32
recursive residuals, whose rounding differs between the kernel's fp64 sums of fp32
values in its own order and the oracle's index-order sums), updates within 2 (reliable
updates) or refinement steps within 1 (restarting); where one of the oracle's
refinement steps ended within a factor 2 of tol, the two sides may stop one step
apart, so one more step and one inner solve's iterations are allowed; the fp64 true relative residual of
each returned x, recomputed by the oracle, <= tol and equal to the reported one to 1e-6
relative; ||x - x_oracle|| / ||x_oracle|| <= 1e-4.  The schedule must not change the
answer: results are compared bit for bit across grid sizes.
"""
import json
import math
import os

import numpy as np
import pytest

import cgproblems as gen
import oracle
from helpers import random_graph_spd, spd_from_pattern, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_2608_09647_gb300 as cg  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch512_ru_oracle.json")


def mixed_systems():
    """Uneven sizes (1 row to several tiles, ragged tails), 5- and 9-point anisotropic
    Laplacians (diagonal layout), a variable diagonal, random row lengths (sliced ELL)."""
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


def rhs(systems, seed=0):
    return [oracle.spmv(A, gen.xstar(A.n, seed + i)) for i, A in enumerate(systems)]


def batch_solve(h, bs, tol, maxit, precond, precision):
    bd = [torch.from_numpy(np.ascontiguousarray(b)).cuda() for b in bs]
    xd = [torch.zeros_like(b) for b in bd]
    st, its, rels = cg.cg_solve_batch(h, bd, xd, tol, maxit, precond, precision)
    torch.cuda.synchronize()
    per = [cg.cg_batch_get_system(h, s) for s in range(len(bs))]
    return st, its, rels, [x.cpu().numpy() for x in xd], per


def make_batch(systems):
    dev = [to_device(A) for A in systems]
    h = cg.cg_batch_create([d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev])
    return h, dev


def oracle_solve(A, b, tol, maxit, precond, precision):
    pc = 1 if precond == cg.CG_PRECOND_JACOBI else 0
    if precision == cg.CG_PREC_FP32_RU:
        return oracle.pcg_ru(A, b, tol=tol, tol_in=0.1, maxit=maxit, max_updates=30, precond=pc)
    return oracle.pcg_ir(A, b, tol=tol, tol_in=1e-4, maxit=maxit, max_outer=30, precond=pc)


def borderline(ref, tol):
    """A refinement step of the oracle ended within a factor 2 of tol: there the two sides
    may stop one step apart, and their inner counts then differ by one inner solve."""
    h = ref.outer_hist if ref.outer_hist is not None else []
    return any(tol / 2 <= v <= 2 * tol for v in h)


def check_system(A, b, its, rel, x, per, ref, tol, precision):
    assert per["status"] == ref.status, (A.name, per, ref.status)
    band = max(5, math.ceil(0.1 * ref.iters))
    upd = 2 if precision == cg.CG_PREC_FP32_RU else 1
    if borderline(ref, tol):
        band += math.ceil(1.5 * ref.iters / max(1, ref.restarts))
        upd += 1
    assert abs(its - ref.iters) <= band, (A.name, its, ref.iters)
    assert abs(per["restarts"] - ref.restarts) <= upd, (A.name, per["restarts"], ref.restarts)
    if np.linalg.norm(b) == 0:
        assert np.all(x == 0) and its == 0
        return
    rel_or = oracle.true_relres(A, b, x)
    if ref.status == cg.CG_OK:
        assert rel_or <= tol * (1 + 1e-6), (A.name, rel_or)
        assert np.linalg.norm(x - ref.x) <= 1e-4 * np.linalg.norm(ref.x), A.name
    assert abs(rel - rel_or) <= 1e-6 * rel_or + 1e-15, (A.name, rel, rel_or)


@pytest.mark.parametrize("precision", [cg.CG_PREC_FP32_RU, cg.CG_PREC_FP32_IR], ids=["ru", "ir"])
@pytest.mark.parametrize("precond", [cg.CG_PRECOND_JACOBI, cg.CG_PRECOND_NONE], ids=["jacobi", "none"])
def test_mixed_fp32_batch_matches_oracle_per_system(precond, precision):
    systems = mixed_systems()
    bs = rhs(systems)
    h, _ = make_batch(systems)
    st, its, rels, xs, per = batch_solve(h, bs, 1e-8, 20000, precond, precision)
    assert st == cg.CG_OK, cg.cg_last_error(h)
    for s, A in enumerate(systems):
        ref = oracle_solve(A, bs[s], 1e-8, 20000, precond, precision)
        check_system(A, bs[s], its[s], rels[s], xs[s], per[s], ref, 1e-8, precision)
    info = cg.cg_get_solve_info(h)
    assert info["iters"] == max(its) and info["kernel_launches"] >= 1
    cg.cg_destroy(h)


def test_reliable_updates_need_fewer_inner_iterations_than_restarting():
    systems = [gen.lap2d(120, 5, 1e-2), gen.lap2d(90, 9, 0.1), gen.diff3d27(12, 1.0, 2)]
    bs = rhs(systems, 3)
    h, _ = make_batch(systems)
    ru = batch_solve(h, bs, 1e-9, 20000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_RU)
    ir = batch_solve(h, bs, 1e-9, 20000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_IR)
    f64 = batch_solve(h, bs, 1e-9, 20000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP64)
    assert ru[0] == ir[0] == f64[0] == cg.CG_OK
    for k_ru, k_ir, k64 in zip(ru[1], ir[1], f64[1]):
        assert k_ru < k_ir
        assert k_ru <= 1.2 * k64 + 5        # the carried direction tracks fp64 PCG's count
    cg.cg_destroy(h)


def test_fp32_schedule_does_not_change_the_answer():
    systems = mixed_systems()
    bs = rhs(systems, 7)
    h, _ = make_batch(systems)
    outs = []
    for grid in (0, 7, 152):
        assert cg.cg_set_option(h, cg.CG_OPT_GRID_CTAS, grid) == cg.CG_OK
        for mode in (1, 2):
            assert cg.cg_set_option(h, cg.CG_OPT_LOOP_MODE, mode) == cg.CG_OK
            outs.append(batch_solve(h, bs, 1e-8, 20000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_RU))
    for o in outs[1:]:
        assert o[1] == outs[0][1] and o[2] == outs[0][2]
        for x, x0 in zip(o[3], outs[0][3]):
            assert np.array_equal(x, x0)
    tune = cg.cg_batch_get_tuning(h, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_RU)
    assert tune["chosen"] >= 0 and len(tune["grids"]) >= 1
    cg.cg_destroy(h)


def test_fp32_batch_edge_cases():
    """b = 0 (x = 0, no iterations), an indefinite system that breaks down (its status,
    the others unaffected), the inner-iteration cap and the update cap."""
    good = gen.lap2d(25, 9, 0.05)
    indef = gen.CSR(2, np.array([0, 1, 2], np.int32), np.array([0, 1], np.int32), np.array([1.0, -1.0]),
                    "indefinite")
    systems = [good, gen.lap2d(10), indef, gen.lap2d(40, 5, 2e-3)]
    bs = rhs(systems, 11)
    bs[1] = np.zeros(systems[1].n)
    bs[2] = np.array([1.0, 1.0])
    h, _ = make_batch(systems)
    st, its, rels, xs, per = batch_solve(h, bs, 1e-8, 20000, cg.CG_PRECOND_NONE, cg.CG_PREC_FP32_RU)
    assert st == cg.CG_ERR_BREAKDOWN
    for s, A in enumerate(systems):
        ref = oracle_solve(A, bs[s], 1e-8, 20000, cg.CG_PRECOND_NONE, cg.CG_PREC_FP32_RU)
        assert per[s]["status"] == ref.status, (A.name, per[s], ref.status)
    assert per[1]["status"] == cg.CG_OK and its[1] == 0 and np.all(xs[1] == 0)
    assert per[2]["status"] == cg.CG_ERR_BREAKDOWN
    for s in (0, 3):
        ref = oracle_solve(systems[s], bs[s], 1e-8, 20000, cg.CG_PRECOND_NONE, cg.CG_PREC_FP32_RU)
        check_system(systems[s], bs[s], its[s], rels[s], xs[s], per[s], ref, 1e-8, cg.CG_PREC_FP32_RU)
    cg.cg_destroy(h)
    # caps: 30 inner iterations in all, then 2 updates at most
    systems = [gen.lap2d(60, 5, 1e-2), gen.lap2d(30, 9, 0.2)]
    bs = rhs(systems, 2)
    h, _ = make_batch(systems)
    st, its, rels, xs, per = batch_solve(h, bs, 1e-8, 30, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_RU)
    assert st == cg.CG_NOT_CONVERGED
    assert all(p["status"] == cg.CG_NOT_CONVERGED and p["iters"] <= 30 for p in per)
    assert cg.cg_set_option(h, cg.CG_OPT_IR_MAX_OUTER, 2) == cg.CG_OK
    st, its, rels, xs, per = batch_solve(h, bs, 1e-12, 20000, cg.CG_PRECOND_JACOBI, cg.CG_PREC_FP32_RU)
    assert st == cg.CG_NOT_CONVERGED and all(p["restarts"] <= 2 for p in per)
    for s, A in enumerate(systems):
        ref = oracle.pcg_ru(A, bs[s], tol=1e-12, tol_in=0.1, maxit=20000, max_updates=2, precond=1)
        assert per[s]["status"] == ref.status and per[s]["restarts"] == ref.restarts
    cg.cg_destroy(h)


def test_full_512_fp32_batch_against_golden_oracle_counts():
    """The 512-system batch workload (as bench.py's batch512_fp32) in one launch against
    the oracle's own reliable-update counts for every member (tests/golden/
    batch512_ru_oracle.json, written from oracle/ alone); every returned x must meet the
    tolerance by the oracle's fp64 residual."""
    if not os.path.exists(GOLDEN):
        pytest.skip("golden fp32 batch counts not generated")
    gold = json.load(open(GOLDEN))
    params = gen.batch_members(512, 0)
    systems = [gen.lap2d(s, p, e) for s, p, e in params]
    bs = [oracle.spmv(A, gen.xstar(A.n, i)) for i, A in enumerate(systems)]
    h, _ = make_batch(systems)
    st, its, rels, xs, per = batch_solve(h, bs, gold["tol"], gold["maxit"], cg.CG_PRECOND_JACOBI,
                                         cg.CG_PREC_FP32_RU)
    assert st == cg.CG_OK, cg.cg_last_error(h)
    for i, (A, m) in enumerate(zip(systems, gold["members"])):
        assert per[i]["status"] == m["status"] == cg.CG_OK
        assert abs(its[i] - m["iters"]) <= max(5, math.ceil(0.1 * m["iters"])), (i, its[i], m["iters"])
        assert abs(per[i]["restarts"] - m["updates"]) <= 2, (i, per[i]["restarts"], m["updates"])
        assert rels[i] <= gold["tol"]
    # the true residual of a sample of members recomputed by the oracle
    for i in range(0, 512, 37):
        assert oracle.true_relres(systems[i], bs[i], xs[i]) <= gold["tol"] * (1 + 1e-6), i
    cg.cg_destroy(h)
