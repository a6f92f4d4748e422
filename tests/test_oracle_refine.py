"""Pins of the reliable-update refinement (reading R8, oracle.pcg_ru / fsai.pcg_ir(carry=True)).

Carrying the search direction over each fp64 update must keep the iteration count
within 20 % of fp64 PCG's, where the restarting refinement (R6) pays a new Krylov build-up
per outer step; both must reach the fp64 tolerance.  A planted mistake in the carry
(a wrong beta) must break the first property.  CPU only."""
import numpy as np
import pytest

import cgproblems as gen
import oracle
from oracle import fsai

MATS = [("q1_48", lambda: gen.q1aniso(48, 1.5, 0.7, 0.01, 3)),
        ("lap9_50", lambda: gen.lap2d(50, 9, 1e-3)),
        ("diff27_14", lambda: gen.diff3d27(14, 1.0, 2))]


@pytest.mark.parametrize("name,make", MATS, ids=[m[0] for m in MATS])
def test_reliable_updates_track_fp64_iterations(name, make):
    A = make()
    b = oracle.spmv(A, gen.xstar(A.n, 4))
    tol = 1e-9
    f64 = oracle.pcg(A, b, tol=tol, maxit=100000, precond=1)
    ir = oracle.pcg_ir(A, b, tol=tol, tol_in=1e-4, maxit=100000, precond=1)
    ru = oracle.pcg_ru(A, b, tol=tol, tol_in=1e-2, maxit=100000, precond=1)
    for s in (f64, ir, ru):
        assert s.status == oracle.OK and oracle.true_relres(A, b, s.x) <= tol * (1 + 1e-9)
    assert ru.iters <= 1.2 * f64.iters + 3, (ru.iters, f64.iters)
    assert ru.iters <= ir.iters
    assert ru.restarts >= 2          # several fp64 updates happened
    # every update contracts the true residual by about the threshold
    h = ru.outer_hist
    assert np.all(h[1:-1] <= 0.1 * h[:-2] + 1e-300)


def test_reliable_updates_with_fsai():
    A = gen.q1aniso(48, 1.5, 2.1, 0.02, 7)
    g = fsai.classic(A)
    b = oracle.spmv(A, gen.xstar(A.n, 5))
    f64 = fsai.pcg(A, g, b, tol=1e-9, maxit=100000)
    ir = fsai.pcg_ir(A, g, b, tol=1e-9, tol_in=1e-4)
    ru = fsai.pcg_ir(A, g, b, tol=1e-9, tol_in=1e-2, carry=True)
    assert f64.status == ir.status == ru.status == oracle.OK
    assert ru.iters <= 1.2 * f64.iters + 3 and ru.iters <= ir.iters
    assert oracle.true_relres(A, b, ru.x) <= 1e-9


def test_a_wrong_carry_is_caught(tmp_path):
    """Plant beta0 = rho_k / rho' (inverted) in a copy of the oracle: the carried
    direction then degrades convergence and the iteration pin fails."""
    import ctypes
    import subprocess
    src = open(oracle._SRC).read()
    old = "const float beta0 = (float)(rho / *rho_io);\n    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta0 * p[i];"
    a = src.index("static int32_t pcg32(")      # the Jacobi inner solve (the first of two sites)
    assert src.index(old) > a and src.count(old) == 2
    bad = src.replace(old, "const float beta0 = (float)(*rho_io / rho);\n    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta0 * p[i];", 1)
    c = tmp_path / "m.c"
    so = tmp_path / "m.so"
    c.write_text(bad)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11", "-o", str(so), str(c), "-lm"],
                   check=True)
    saved = oracle._lib
    oracle._lib = oracle._bind(ctypes.CDLL(str(so)))
    try:
        A = gen.q1aniso(48, 1.5, 0.7, 0.01, 3)
        b = oracle.spmv(A, gen.xstar(A.n, 4))
        f64 = oracle.pcg(A, b, tol=1e-9, maxit=100000, precond=1)
        ru = oracle.pcg_ru(A, b, tol=1e-9, tol_in=1e-2, maxit=100000, precond=1)
        assert not (ru.status == oracle.OK and ru.iters <= 1.2 * f64.iters + 3)
    finally:
        oracle._lib = saved
