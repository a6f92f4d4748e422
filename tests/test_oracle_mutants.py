"""Plant plausible mistakes in a copy of the oracle source (on the CPU) and check that
the pins catch each one: a flipped sign, a dropped term, a wrong index, swapped
operands and a dropped preconditioner must all fail at least one pin."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.linalg

import cgproblems as gen
import oracle
from test_oracle_pins import csr_from_scipy, random_spd, cheb_iters

MUTANTS = {
    "spmv_wrong_index": ("s += vals[k] * x[colind[k]];\n    y[i] = s;",
                         "s += vals[k] * x[i];\n    y[i] = s;"),
    "r_update_sign": ("      for (int64_t i = 0; i < n; ++i) r[i] -= alpha * q[i];",
                      "      for (int64_t i = 0; i < n; ++i) r[i] += alpha * q[i];"),
    "beta_swapped": ("const double beta = rho_new / rho;", "const double beta = rho / rho_new;"),
    "p_update_dropped_term": ("      for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];",
                              "      for (int64_t i = 0; i < n; ++i) p[i] = z[i];"),
    "x_update_uses_q": ("x[i] += alpha * p[i];", "x[i] += alpha * q[i];"),
    "jacobi_dropped": ("z[i] = precond ? r[i] * dinv[i] : r[i];\n      const double rho_new",
                       "z[i] = r[i];\n      const double rho_new"),
}


def _pins_pass(lib) -> bool:
    saved = oracle._lib
    oracle._lib = lib
    try:
        checks = []
        A = gen.lap2d(9)
        x = gen.xstar(A.n, 1)
        checks.append(np.allclose(oracle.spmv(A, x), A.to_scipy() @ x, rtol=1e-13, atol=1e-13))
        for precond in (0, 1):
            Ad = random_spd(32, 100.0, 1)
            b = np.random.default_rng(5).standard_normal(32)
            s = oracle.pcg(csr_from_scipy(Ad), b, tol=1e-10, maxit=320, precond=precond)
            xc = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Ad), b)
            checks.append(s.status == 0 and
                          np.linalg.norm(s.x - xc) <= 1e-6 * np.linalg.norm(xc))
        A = gen.lap2d(24)
        b = oracle.spmv(A, gen.xstar(A.n, 0))
        s = oracle.pcg(A, b, tol=1e-8, maxit=1000, precond=0)
        kappa = 1.0 / np.tan(np.pi / 50) ** 2
        checks.append(s.status == 0 and s.iters <= cheb_iters(kappa, 1e-8))
        # Jacobi-PCG equals CG on the symmetrically scaled system
        rng = np.random.default_rng(12)
        Ad = random_spd(30, 50.0, 12)
        Dh = np.diag(rng.uniform(0.3, 4.0, 30))
        Ad = Dh @ Ad @ Dh
        b = rng.standard_normal(30)
        si = 1.0 / np.sqrt(np.diag(Ad))
        s1 = oracle.pcg(csr_from_scipy(Ad), b, tol=0.0, maxit=8, precond=1, max_restarts=0)
        s0 = oracle.pcg(csr_from_scipy(Ad * np.outer(si, si)), si * b, tol=0.0, maxit=8,
                        precond=0, max_restarts=0)
        checks.append(np.linalg.norm(s1.x - si * s0.x) <= 1e-10 * np.linalg.norm(si * s0.x))
        return all(checks)
    finally:
        oracle._lib = saved


def _build_variant(tmp_path, src_text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    so = tmp_path / f"liboracle_{tag}.so"
    src.write_text(src_text)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-std=c11",
                    "-o", str(so), str(src), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    return oracle._bind(lib)


def test_unmutated_copy_passes(tmp_path):
    text = open(oracle._SRC).read()
    assert _pins_pass(_build_variant(tmp_path, text, "clean"))


def _pcg_body(text):
    """Span of or_pcg (the function these mutants target) in the oracle source."""
    a = text.index("\nint or_pcg(")
    b = text.index("\n}\n", a) + 3
    return a, b


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(oracle._SRC).read()
    if name == "spmv_wrong_index":  # or_spmv, ahead of or_pcg
        a, b = 0, text.index("\nint or_pcg(")
    else:
        a, b = _pcg_body(text)
    body = text[a:b]
    assert body.count(old) == 1, f"mutation site for {name} not unique"
    text = text[:a] + body.replace(old, new) + text[b:]
    assert not _pins_pass(_build_variant(tmp_path, text, name))


# Mistakes in the FSAI application z = G^T (G r) (fsai_apply, the fp64 one): the second
# factor applied untransposed (z = G G r, a transposed operand) or dropped (z = G r).
FSAI_MUTANTS = {
    "fsai_second_factor_untransposed": (
        "    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) z[gci[k]] += gval[k] * t[i];",
        "    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) z[i] += gval[k] * t[gci[k]];"),
    "fsai_second_factor_dropped": (
        "    for (int64_t k = grp[i]; k < grp[i + 1]; ++k) z[gci[k]] += gval[k] * t[i];",
        "    z[i] = t[i];"),
}


def _fsai_pins_pass(lib) -> bool:
    """The dense-pattern pin: classic FSAI of a dense SPD matrix (numpy, independent of
    the C code) is the inverse Cholesky factor, so FSAI-PCG converges in one iteration."""
    from oracle import fsai
    saved = fsai._load
    fsai._load = lambda: lib
    try:
        M = random_spd(12, 100.0, 3)
        A = csr_from_scipy(M)
        g = fsai.classic(A)
        b = M @ np.ones(12)
        s = fsai.pcg(A, g, b, tol=1e-12, maxit=50)
        return s.status == oracle.OK and s.iters == 1 and np.allclose(s.x, np.ones(12), atol=1e-9)
    finally:
        fsai._load = saved


def _fsai_apply_body(text):
    a = text.index("static void fsai_apply(")
    b = text.index("\n}\n", a) + 3
    return a, b


def test_unmutated_copy_passes_the_fsai_pin(tmp_path):
    assert _fsai_pins_pass(_build_variant(tmp_path, open(oracle._SRC).read(), "clean_fsai"))


@pytest.mark.parametrize("name", sorted(FSAI_MUTANTS))
def test_fsai_mutant_is_caught(tmp_path, name):
    old, new = FSAI_MUTANTS[name]
    text = open(oracle._SRC).read()
    a, b = _fsai_apply_body(text)
    body = text[a:b]
    assert body.count(old) == 1, f"mutation site for {name} not unique"
    text = text[:a] + body.replace(old, new) + text[b:]
    assert not _fsai_pins_pass(_build_variant(tmp_path, text, name))
