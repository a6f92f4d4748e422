"""Pins for the fp64 oracle against facts fixed outside the oracle itself:
closed-form eigenpairs of the Dirichlet Laplacians, dense Cholesky, finite
termination of CG, A-orthogonality of the search directions, the Chebyshev
iteration bound, and the special cases of the method (b = 0, constant
diagonal, indefinite matrices).  None of these re-types the oracle's formulas.

Paper anchors: CSR SpMV, Sec. 3.1; CG iteration, Alg. 1; fp64, Sec. 3.1.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp

import cgproblems as gen
import oracle


def csr_from_scipy(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return gen.CSR(M.shape[0], M.indptr.astype(np.int32), M.indices.astype(np.int32),
                   M.data.astype(np.float64), "scipy")


def random_spd(n, kappa, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, kappa, n)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


def cheb_iters(kappa, tol):
    """Smallest k with 2 sqrt(kappa) ((sqrt(kappa)-1)/(sqrt(kappa)+1))^k <= tol, a bound on
    ||r_k||/||r_0|| for CG (from the A-norm bound and ||r|| <= sqrt(kappa) ||e||_A scaling)."""
    s = math.sqrt(kappa)
    return math.ceil(math.log(tol / (2.0 * s)) / math.log((s - 1.0) / (s + 1.0)))


# ---------------------------------------------------------------- SpMV pins

@pytest.mark.parametrize("A", [gen.lap2d(17), gen.lap2d(9, 9, 0.01), gen.lap3d7(7),
                               gen.diff3d27(6, 1.0, 4), gen.q1aniso(11, 1.5, 0.4, 0.02, 9)],
                         ids=lambda A: A.name)
def test_spmv_matches_scipy(A):
    x = gen.xstar(A.n, 11)
    y = oracle.spmv(A, x)
    ref = A.to_scipy() @ x
    scale = np.abs(A.to_scipy()) @ np.abs(x)
    assert np.all(np.abs(y - ref) <= 1e-14 * scale)


def test_spmv_ones_gives_boundary_weights_2d():
    """A 1: zero in the interior, the number of missing neighbours on the boundary (stencil 4,-1)."""
    N = 12
    y = oracle.spmv(gen.lap2d(N), np.ones(N * N)).reshape(N, N)
    expect = np.zeros((N, N))
    expect[0, :] += 1
    expect[-1, :] += 1
    expect[:, 0] += 1
    expect[:, -1] += 1
    assert np.array_equal(y, expect)


def test_spmv_ones_gives_boundary_weights_27pt():
    """Row sums of the 27-point graph Laplacian equal the weights of the ghost edges only,
    so they vanish exactly for interior rows and are positive on the boundary."""
    N = 6
    A = gen.diff3d27(N, 1.0, 2)
    y = oracle.spmv(A, np.ones(A.n)).reshape(N, N, N)
    interior = y[1:-1, 1:-1, 1:-1]
    assert np.all(np.abs(interior) <= 1e-12 * np.abs(A.vals).max())
    mask = np.ones((N, N, N), bool)
    mask[1:-1, 1:-1, 1:-1] = False
    assert np.all(y[mask] > 0)


@pytest.mark.parametrize("N,j,k", [(9, 1, 1), (9, 3, 7), (16, 2, 15), (31, 5, 5)])
def test_spmv_sine_mode_2d(N, j, k):
    """The 5-point Dirichlet Laplacian maps the sine mode (j, k) to lambda_jk times itself,
    lambda_jk = 4 sin^2(j pi / 2(N+1)) + 4 sin^2(k pi / 2(N+1))."""
    i = np.arange(1, N + 1)
    vx = np.sin(j * np.pi * i / (N + 1))
    vy = np.sin(k * np.pi * i / (N + 1))
    v = np.outer(vy, vx).ravel()  # row index y*N + x
    lam = 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2 + 4 * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    y = oracle.spmv(gen.lap2d(N), v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13


@pytest.mark.parametrize("eps", [1.0, 0.1, 1e-3])
def test_spmv_sine_mode_2d_anisotropic(eps):
    N, j, k = 13, 2, 9
    i = np.arange(1, N + 1)
    v = np.outer(np.sin(k * np.pi * i / (N + 1)), np.sin(j * np.pi * i / (N + 1))).ravel()
    lam = eps * 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2 + 4 * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    y = oracle.spmv(gen.lap2d(N, 5, eps), v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13


def test_spmv_sine_mode_3d():
    N, (a, b_, c) = 10, (1, 4, 9)
    i = np.arange(1, N + 1)
    s = lambda m: np.sin(m * np.pi * i / (N + 1))
    v = np.einsum("z,y,x->zyx", s(c), s(b_), s(a)).ravel()
    lam = sum(4 * np.sin(m * np.pi / (2 * (N + 1))) ** 2 for m in (a, b_, c))
    y = oracle.spmv(gen.lap3d7(N), v)
    assert np.max(np.abs(y - lam * v)) <= 1e-13


# ---------------------------------------------------------------- CG pins

@pytest.mark.parametrize("n,kappa,seed", [(8, 10, 0), (32, 1e2, 1), (64, 1e3, 2), (50, 5e2, 3)])
@pytest.mark.parametrize("precond", [0, 1])
def test_cg_matches_dense_cholesky(n, kappa, seed, precond):
    Ad = random_spd(n, kappa, seed)
    A = csr_from_scipy(Ad)
    b = np.random.default_rng(seed + 100).standard_normal(n)
    tol = 1e-10
    s = oracle.pcg(A, b, tol=tol, maxit=10 * n, precond=precond)
    xc = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Ad), b)
    assert s.status == oracle.OK
    assert s.relres_true <= tol
    assert np.linalg.norm(s.x - xc) / np.linalg.norm(xc) <= kappa * tol * 10


@pytest.mark.parametrize("n,seed", [(16, 5), (40, 6), (64, 7)])
def test_cg_terminates_within_n_iterations(n, seed):
    """Finite termination: at most n steps on a well-conditioned n x n SPD system."""
    A = csr_from_scipy(random_spd(n, 5.0, seed))
    b = np.random.default_rng(seed).standard_normal(n)
    s = oracle.pcg(A, b, tol=1e-12, maxit=n, precond=0, max_restarts=0)
    assert s.status == oracle.OK
    assert s.iters <= n


@pytest.mark.parametrize("m", [1, 2, 5, 9])
def test_cg_1d_poisson_m_eigenvectors_in_m_steps(m):
    """b spanned by m eigenvectors of the 1-D Poisson matrix (distinct eigenvalues):
    the Krylov space closes after m steps, so CG drops from O(1) to rounding level (here
    below 1e-9; the sines carry ~1e-16 of every other mode) in exactly m iterations."""
    n = 60
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    A = csr_from_scipy(T)
    i = np.arange(1, n + 1)
    modes = [3, 7, 11, 20, 29, 33, 41, 50, 57][:m]
    b = sum((jj + 1.0) * np.sin(mode * np.pi * i / (n + 1)) for jj, mode in enumerate(modes))
    s = oracle.pcg(A, b, tol=1e-9, maxit=n, precond=0, max_restarts=0, res_hist=True)
    assert s.status == oracle.OK
    assert s.iters == m
    if m > 1:
        assert s.res_hist[m - 1] > 1e-3  # not converged one step earlier


def test_search_directions_are_A_orthogonal():
    Ad = random_spd(60, 50.0, 9)
    A = csr_from_scipy(Ad)
    b = np.random.default_rng(9).standard_normal(60)
    s = oracle.pcg(A, b, tol=1e-14, maxit=60, precond=0, max_restarts=0, p_hist_k=10)
    P = s.p_hist
    G = P @ Ad @ P.T
    nrm = np.sqrt(np.diag(G))
    off = np.abs(G) / np.outer(nrm, nrm)
    np.fill_diagonal(off, 0.0)
    assert off.max() <= 1e-10


def test_search_directions_are_A_orthogonal_jacobi():
    """With M = D, the directions stay A-orthogonal (PCG is CG on D^-1/2 A D^-1/2)."""
    rng = np.random.default_rng(3)
    Ad = random_spd(48, 30.0, 4)
    Dh = np.diag(rng.uniform(0.5, 3.0, 48))
    Ad = Dh @ Ad @ Dh
    A = csr_from_scipy(Ad)
    s = oracle.pcg(A, rng.standard_normal(48), tol=1e-14, maxit=48, precond=1,
                   max_restarts=0, p_hist_k=10)
    P = s.p_hist
    G = P @ Ad @ P.T
    nrm = np.sqrt(np.diag(G))
    off = np.abs(G) / np.outer(nrm, nrm)
    np.fill_diagonal(off, 0.0)
    assert off.max() <= 1e-10


@pytest.mark.parametrize("N", [16, 32, 64])
def test_cg_iterations_below_chebyshev_bound_2d(N):
    """kappa of the 5-point Laplacian is cot^2(pi / 2(N+1)); the oracle must need no more
    iterations than the Chebyshev bound (473 at N = 64, tol 1e-8)."""
    A = gen.lap2d(N)
    b = oracle.spmv(A, gen.xstar(A.n, 0))
    kappa = 1.0 / math.tan(math.pi / (2 * (N + 1))) ** 2
    s = oracle.pcg(A, b, tol=1e-8, maxit=1000, precond=0)
    assert s.status == oracle.OK
    assert s.iters <= cheb_iters(kappa, 1e-8)
    if N == 64:
        assert cheb_iters(kappa, 1e-8) == 473


def test_cg_iterations_below_chebyshev_bound_3d():
    N = 20
    A = gen.lap3d7(N)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    kappa = 1.0 / math.tan(math.pi / (2 * (N + 1))) ** 2
    s = oracle.pcg(A, b, tol=1e-8, maxit=2000, precond=1)
    assert s.status == oracle.OK
    assert s.iters <= cheb_iters(kappa, 1e-8)


def test_chebyshev_bound_values_for_the_workloads():
    """The bounds quoted for the workloads: 256^3 7-point -> 1981 iterations."""
    assert cheb_iters(1.0 / math.tan(math.pi / 514) ** 2, 1e-8) == 1981


def test_residual_history_is_rate_bounded():
    """||r_k|| / ||r_0|| <= 2 sqrt(kappa) rho^k at every step for the 2-D Laplacian."""
    N = 24
    A = gen.lap2d(N)
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    kappa = 1.0 / math.tan(math.pi / (2 * (N + 1))) ** 2
    s = oracle.pcg(A, b, tol=1e-10, maxit=1000, precond=0, res_hist=True)
    rate = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    k = np.arange(len(s.res_hist))
    assert np.all(s.res_hist / s.res_hist[0] <= 2 * math.sqrt(kappa) * rate ** k * (1 + 1e-9))


def test_jacobi_equals_cg_for_constant_diagonal():
    """With a constant diagonal, M = cI and Jacobi-PCG is CG step for step."""
    for A in (gen.lap3d7(9), gen.lap2d(20, 5, 0.3)):
        b = oracle.spmv(A, gen.xstar(A.n, 5))
        s0 = oracle.pcg(A, b, tol=1e-9, maxit=1000, precond=0)
        s1 = oracle.pcg(A, b, tol=1e-9, maxit=1000, precond=1)
        assert s0.iters == s1.iters
        assert np.max(np.abs(s0.x - s1.x)) <= 1e-12 * np.max(np.abs(s0.x))


def test_solution_error_against_known_xstar():
    A = gen.lap2d(32)
    xs = gen.xstar(A.n, 7)
    b = oracle.spmv(A, xs)
    s = oracle.pcg(A, b, tol=1e-12, maxit=2000, precond=1)
    kappa = 1.0 / math.tan(math.pi / 66) ** 2
    assert s.relres_true <= 1e-12
    assert np.linalg.norm(s.x - xs) / np.linalg.norm(xs) <= kappa * 1e-12


# ---------------------------------------------------------------- special cases

def test_zero_rhs_returns_zero():
    A = gen.lap2d(8)
    s = oracle.pcg(A, np.zeros(A.n), x0=np.ones(A.n), tol=1e-8, maxit=100)
    assert s.status == oracle.OK and s.iters == 0 and np.all(s.x == 0)


def test_exact_initial_guess_takes_zero_iterations():
    A = gen.lap2d(8)
    xs = gen.xstar(A.n, 3)
    b = oracle.spmv(A, xs)
    s = oracle.pcg(A, b, x0=xs, tol=1e-8, maxit=100)
    assert s.status == oracle.OK and s.iters == 0


def test_indefinite_matrix_breaks_down():
    Ad = np.diag([1.0, 2.0, -3.0, 4.0])
    A = csr_from_scipy(Ad)
    s = oracle.pcg(A, np.ones(4), tol=1e-10, maxit=10, precond=0)
    assert s.status == oracle.ERR_BREAKDOWN


def test_nan_rhs_is_numeric_error():
    A = gen.lap2d(6)
    b = np.ones(A.n)
    b[5] = np.nan
    s = oracle.pcg(A, b, tol=1e-8, maxit=10)
    assert s.status == oracle.ERR_NUMERIC


def test_maxit_reports_not_converged():
    A = gen.lap2d(32)
    b = oracle.spmv(A, gen.xstar(A.n, 1))
    s = oracle.pcg(A, b, tol=1e-12, maxit=10)
    assert s.status == oracle.NOT_CONVERGED and s.iters == 10
    assert s.relres_true > 1e-12


def test_jacobi_rejects_nonpositive_diagonal():
    A = csr_from_scipy(np.array([[1.0, 0.5], [0.5, -1.0]]))
    assert oracle.pcg(A, np.ones(2), precond=1).status == oracle.ERR_INVALID


# ---------------------------------------------------------------- mixed precision

@pytest.mark.parametrize("tol_in", [1e-3, 1e-4, 1e-5])
def test_refinement_reaches_fp64_tolerance(tol_in):
    A = gen.diff3d27(10, 1.0, 3)
    xs = gen.xstar(A.n, 3)
    b = oracle.spmv(A, xs)
    s = oracle.pcg_ir(A, b, tol=1e-10, tol_in=tol_in)
    ref = oracle.pcg(A, b, tol=1e-12, maxit=5000)
    assert s.status == oracle.OK
    assert s.relres_true <= 1e-10
    # each refinement step contracts the fp64 residual by about tol_in
    h = s.outer_hist
    assert np.all(h[1:] <= h[:-1] * max(10 * tol_in, 1e-2))
    assert np.linalg.norm(s.x - ref.x) / np.linalg.norm(ref.x) <= 1e-8


def test_refinement_fp32_floor_does_not_stall():
    """An inner tolerance below the fp32 floor still converges in fp64 via refinement."""
    A = gen.lap2d(40)
    b = oracle.spmv(A, gen.xstar(A.n, 4))
    s = oracle.pcg_ir(A, b, tol=1e-12, tol_in=1e-7, maxit=20000)
    assert s.status == oracle.OK and s.relres_true <= 1e-12


def test_jacobi_pcg_is_cg_on_the_symmetrically_scaled_system():
    """Jacobi-PCG on A is CG on D^-1/2 A D^-1/2 with b^ = D^-1/2 b and x = D^-1/2 x^:
    after the same number of steps the iterates agree (scaling built here with numpy)."""
    rng = np.random.default_rng(12)
    Ad = random_spd(40, 50.0, 12)
    Dh = np.diag(rng.uniform(0.3, 4.0, 40))
    Ad = Dh @ Ad @ Dh
    b = rng.standard_normal(40)
    s_inv = 1.0 / np.sqrt(np.diag(Ad))
    Ah = Ad * np.outer(s_inv, s_inv)
    for k in (3, 8, 15):
        s1 = oracle.pcg(csr_from_scipy(Ad), b, tol=0.0, maxit=k, precond=1, max_restarts=0)
        s0 = oracle.pcg(csr_from_scipy(Ah), s_inv * b, tol=0.0, maxit=k, precond=0,
                        max_restarts=0)
        assert s1.iters == s0.iters == k
        x_scaled = s_inv * s0.x
        assert np.linalg.norm(s1.x - x_scaled) <= 1e-10 * np.linalg.norm(x_scaled)
