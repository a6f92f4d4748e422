"""Pins of the FSAI oracle (oracle/fsai.py) against facts fixed by the mathematics:
the exact inverse factor on a full pattern, the Kaporin minimiser property, finite
differences, the Jacobi special case, SPD-ness, and hand-checked rounding and
feature values.  CPU only."""
import math

import numpy as np
import pytest

import cgproblems as gen
import oracle
from oracle import fsai


def dense_csr(M, name):
    import scipy.sparse as sp
    S = sp.csr_matrix(M)
    S.sort_indices()
    return gen.CSR(M.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32),
                   S.data.astype(np.float64), name)


def random_spd(n, seed):
    rng = np.random.default_rng(seed)
    B = rng.normal(size=(n, n))
    return B @ B.T + n * np.eye(n)


def test_bf16_rounding_table():
    # 8 significant bits, ties to even
    cases = {1.0: 1.0, 1.0 + 2 ** -8: 1.0, 1.0 + 3 * 2 ** -8: 1.0 + 2 ** -6,
             1.0 + 2 ** -9: 1.0, 1.0 + 2 ** -8 + 2 ** -12: 1.0 + 2 ** -7,
             -3.0: -3.0, 0.0: 0.0, 255.5: 256.0, 254.5: 254.0, 1e-20: 1e-20 * 0 + fsai.bf16(1e-20)}
    for x, want in cases.items():
        assert fsai.bf16(x) == want, (x, fsai.bf16(x), want)
    x = np.random.default_rng(0).normal(size=1000)
    r = fsai.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2 ** -8)
    assert np.array_equal(fsai.bf16(r), r)


def test_full_pattern_gives_the_exact_inverse_factor():
    """On a dense SPD matrix tril(A) is the full lower pattern, so classic FSAI is the
    inverse Cholesky factor: G A G^T = I, and PCG converges in one iteration."""
    M = random_spd(12, 1)
    A = dense_csr(M, "dense12")
    g = fsai.classic(A)
    G = fsai.g_matrix(A, g).toarray()
    assert np.allclose(G @ M @ G.T, np.eye(12), atol=1e-12)
    L = np.linalg.cholesky(M)
    assert np.allclose(G, np.linalg.inv(L), atol=1e-12)
    b = M @ np.ones(12)
    s = fsai.pcg(A, g, b, tol=1e-12, maxit=50)
    assert s.status == oracle.OK and s.iters == 1


@pytest.mark.parametrize("make", [lambda: gen.q1aniso(10, 1.5, 0.7, 0.02, 4),
                                  lambda: gen.lap2d(9, 9, 0.1),
                                  lambda: gen.diff3d27(5, 1.0, 2)])
def test_classic_fsai_minimises_the_kaporin_number(make):
    A = make()
    g = fsai.classic(A)
    G = fsai.g_matrix(A, g)
    S = A.to_scipy()
    assert np.allclose((G @ S @ G.T).diagonal(), 1.0, atol=1e-12)   # normalisation of F2
    L0, dG = fsai.kaporin(A, g)
    assert np.linalg.norm(dG) < 1e-10                                # stationary point
    rng = np.random.default_rng(7)
    for _ in range(20):
        pert = g + 1e-2 * rng.normal(size=g.size) * np.abs(g)
        assert fsai.kaporin(A, pert)[0] > L0
    # scale invariance of the Kaporin number
    assert abs(fsai.kaporin(A, 3.0 * g)[0] - L0) < 1e-12


def fd_check(f, x, grad, idx, h):
    for k in idx:
        e = np.zeros_like(x)
        e[k] = h
        num = (f(x + e) - f(x - e)) / (2 * h)
        assert abs(num - grad[k]) <= 1e-6 * max(1.0, abs(num)) * max(1.0, np.max(np.abs(grad))), \
            (k, num, grad[k])


def test_kaporin_and_residual_gradients_match_finite_differences():
    A = gen.q1aniso(8, 1.5, 1.1, 0.1, 5)
    rng = np.random.default_rng(3)
    g = fsai.classic(A) * (1 + 0.1 * rng.normal(size=len(fsai.tril(A)[1])))
    L, dG = fsai.kaporin(A, g)
    fd_check(lambda v: fsai.kaporin(A, v)[0], g, dG, rng.choice(g.size, 25, replace=False), 1e-6)
    R = rng.normal(size=(3, A.n))
    LR, dR = fsai.residual_term(A, g, R)
    fd_check(lambda v: fsai.residual_term(A, v, R)[0], g, dR, rng.choice(g.size, 25, replace=False), 1e-6)


def test_parameter_gradient_matches_finite_differences():
    """Through features, MLP and the G mapping (fp64 mode, no bf16 rounding)."""
    A = gen.q1aniso(7, 1.5, 0.3, 0.05, 6)
    rng = np.random.default_rng(4)
    p = fsai.init_params(1).astype(np.float64)
    p[-65:] = rng.normal(0, 0.05, 65)   # a non-zero output layer
    R = rng.normal(size=(2, A.n))
    f = lambda v: fsai.loss_and_grad(A, v, R, 0.1, round_bf16=False)[0]
    L, grad = fsai.loss_and_grad(A, p, R, 0.1, round_bf16=False)
    idx = np.concatenate([rng.choice(2048, 12, replace=False),           # W1
                          2048 + 64 + rng.choice(4096, 12, replace=False),  # W2
                          np.arange(6337 - 65, 6337)[rng.choice(65, 10, replace=False)],
                          [2048 + 3, 2048 + 64 + 4096 + 5]])             # b1, b2
    fd_check(f, p, grad, idx, 1e-6)


def test_zero_output_layer_is_jacobi():
    """o = 0 gives G = D^-1/2: the same G, Kaporin value and PCG iterations as Jacobi."""
    A = gen.q1aniso(14, 1.5, 2.0, 0.01, 8)
    p = fsai.init_params(3)
    g = fsai.learned(A, p)
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    jac = np.where(rows == tci, 1.0 / np.sqrt(fsai.diag(A))[rows], 0.0)
    assert np.allclose(g, jac, rtol=0, atol=1e-15 * np.max(jac))
    b = oracle.spmv(A, gen.xstar(A.n, 2))
    s1 = fsai.pcg(A, g, b, tol=1e-9, maxit=2000)
    s2 = oracle.pcg(A, b, tol=1e-9, maxit=2000, precond=1)
    assert s1.status == s2.status == oracle.OK and s1.iters == s2.iters
    # same iterates up to the rounding of r / sqrt(d) / sqrt(d) versus r / d
    assert np.linalg.norm(s1.x - s2.x) <= 1e-7 * np.linalg.norm(s2.x)


def test_learned_factor_is_spd_and_pcg_stays_positive():
    A = gen.q1aniso(10, 1.5, 0.9, 0.2, 9)
    rng = np.random.default_rng(11)
    p = fsai.init_params(5).astype(np.float64)
    p[-65:] = rng.normal(0, 0.05, 65)   # small enough to keep G well conditioned
    g = fsai.learned(A, p)
    G = fsai.g_matrix(A, g).toarray()
    assert np.all(np.diag(G) > 0)
    np.linalg.cholesky(G @ A.to_dense() @ G.T)    # SPD
    b = oracle.spmv(A, gen.xstar(A.n, 4))
    s = fsai.pcg(A, g, b, tol=1e-9, maxit=2000)
    assert s.status == oracle.OK and s.rz_min > 0


def test_features_of_a_constant_laplacian_row():
    """Interior row of the 5-point unit Laplacian on a 6 x 6 grid (row i = 8, x = 2, y = 1)."""
    A = gen.lap2d(6)
    F = fsai.features(A)
    trp, tci, _ = fsai.tril(A)
    i = 8
    rows = F[trp[i]:trp[i + 1]]
    assert list(tci[trp[i]:trp[i + 1]]) == [2, 7, 8]
    # offsets of A: -6, -1, 0, 1, 6 -> tril slots (-6, -1, 0)
    assert np.array_equal(rows[:, 0:8].argmax(1), [0, 1, 2])
    assert np.allclose(rows[:, 8], [-0.25, -0.25, 1.0])
    assert np.allclose(rows[:, 9], 0.0)
    assert np.allclose(rows[0, 10:15], [-0.25, -0.25, 1.0, -0.25, -0.25])
    assert np.allclose(rows[:, 15:19], 0.0) and np.allclose(rows[:, 28], 1.0)
    # row j = 2 (y = 0) lies on the boundary below: no offset -6 entry
    assert np.allclose(rows[0, 19:24], [0.0, -0.25, 1.0, -0.25, -0.25])


def test_adam_first_step_moves_each_parameter_by_lr():
    p = np.zeros(5)
    g = np.array([1.0, -2.0, 1e-3, 0.0, 5.0])
    p1, m, v = fsai.adam(p, g, np.zeros(5), np.zeros(5), 1, lr=0.1)
    assert np.allclose(p1[[0, 1, 2, 4]], -0.1 * np.sign(g[[0, 1, 2, 4]]), rtol=1e-4)
    assert p1[3] == 0.0


def test_fsai_refinement_reaches_tolerance():
    A = gen.q1aniso(16, 1.5, 0.2, 0.01, 12)
    g = fsai.classic(A)
    b = oracle.spmv(A, gen.xstar(A.n, 6))
    s = fsai.pcg_ir(A, g, b, tol=1e-10, tol_in=1e-4)
    assert s.status == oracle.OK and s.relres_true <= 1e-10
    assert oracle.true_relres(A, b, s.x) <= 1e-10


def test_mlp_forward_by_hand():
    """A network small enough to evaluate on paper (F4): every weight a bf16-exact
    number.  Unit 0 of layer 1 reads feature 3 (x2), unit 1 reads feature 7 (x -1, bias
    0.5); unit 0 of layer 2 is h1_0 + 3 h1_1 - 0.25 (an off-diagonal W2 entry, so a
    transposed W2 reads the wrong unit), unit 5 is -h1_1 (never positive: only the
    second ReLU keeps it out); o = 0.5 h2_0 + 4 h2_5 + 0.125."""
    W1 = np.zeros((fsai.N_HID, fsai.N_IN)); b1 = np.zeros(fsai.N_HID)
    W2 = np.zeros((fsai.N_HID, fsai.N_HID)); b2 = np.zeros(fsai.N_HID)
    W3 = np.zeros(fsai.N_HID)
    W1[0, 3], W1[1, 7], b1[1] = 2.0, -1.0, 0.5
    W2[0, 0], W2[0, 1], b2[0], W2[5, 1] = 1.0, 3.0, -0.25, -1.0
    W3[0], W3[5] = 0.5, 4.0
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [0.125]])
    assert all(np.array_equal(u, v) for u, v in zip(fsai.unpack(p), (W1, b1, W2, b2, W3, 0.125)))
    F = np.zeros((3, fsai.N_IN))
    F[0, 3], F[0, 7] = 1.5, 0.25      # h1 = (3, 0.25); z2_0 = 3.5; z2_5 = -0.25
    F[1, 3], F[1, 7] = -1.0, 2.0      # h1 = (0, 0): both first-layer units cut by the ReLU
    F[2, 3], F[2, 7] = 0.25, -0.5     # h1 = (0.5, 1.0); z2_0 = 3.25; z2_5 = -1
    F[:, 0] = 7.0                     # a feature no unit reads
    want = np.array([0.5 * 3.5 + 0.125, 0.125, 0.5 * 3.25 + 0.125])
    for rnd in (True, False):
        o, _ = fsai.mlp_forward(p, F, round_bf16=rnd)
        assert np.array_equal(o, want), (rnd, o, want)


def test_loss_terms_in_closed_form():
    """The Jacobi factor G = D^-1/2 makes every g_i^T A g_i = 1, so the Kaporin term is
    the mean of log A_ii (F6); the exact inverse factor of a dense SPD matrix makes
    G^T G = A^-1, so A G^T G r = r and the residual term vanishes."""
    A = gen.q1aniso(9, 1.5, 0.4, 0.05, 2)
    d = A.to_scipy().diagonal()
    trp, tci, _ = fsai.tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    gj = np.where(tci == rows, 1.0 / np.sqrt(d[rows]), 0.0)
    L, _ = fsai.kaporin(A, gj)
    assert abs(L - np.mean(np.log(d))) <= 1e-13 * abs(np.mean(np.log(d))) + 1e-14
    M = random_spd(10, 4)
    Ad = dense_csr(M, "dense10")
    g = fsai.classic(Ad)
    R = np.random.default_rng(3).standard_normal((3, 10))
    LR, _ = fsai.residual_term(Ad, g, R)
    assert LR <= 1e-24


def hand_network():
    """The network of test_mlp_forward_by_hand: bf16-exact weights."""
    W1 = np.zeros((fsai.N_HID, fsai.N_IN)); b1 = np.zeros(fsai.N_HID)
    W2 = np.zeros((fsai.N_HID, fsai.N_HID)); b2 = np.zeros(fsai.N_HID)
    W3 = np.zeros(fsai.N_HID)
    W1[0, 3], W1[1, 7], b1[1] = 2.0, -1.0, 0.5
    W2[0, 0], W2[0, 1], b2[0], W2[5, 1] = 1.0, 3.0, -0.25, -1.0
    W3[0], W3[5] = 0.5, 4.0
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [0.125]])


D_A = 1.0 + 3 * 2.0 ** -9        # dLoss/do of entry A: not a bf16 value (bf16(D_A) = 1 + 2^-7)


def hand_backward_case():
    """Two entries.  A: x3 = 1.5, x7 = 0.25, x0 = 7 -> z1 = (3, 0.25), z2_0 = 3.5,
    z2_5 = -0.25 (masked; W3_5 = 4 would leak through a missing second-layer mask);
    dout = D_A.  B: x3 = 1.5, x7 = 1 -> z1 = (3, -0.5) (unit 1 cut by the first ReLU,
    yet it receives dh1_1 = 3 dz2_0 through W2[0, 1]), z2_0 = 2.75; dout = 1."""
    F = np.zeros((2, fsai.N_IN))
    F[0, 3], F[0, 7], F[0, 0] = 1.5, 0.25, 7.0
    F[1, 3], F[1, 7] = 1.5, 1.0
    return F, np.array([D_A, 1.0])


def hand_backward_expected(rounded):
    """The gradient worked by hand (F7).  Entry A: dz2_0 = 0.5 D_A = 0.5029296875, which
    bf16 rounds to 0.50390625; dh1 = dz2r_0 (W2[0, 0], W2[0, 1]) = (0.50390625, 1.51171875);
    dz1_1 = 1.51171875 needs 9 significant bits and rounds (tie, to even) to 1.515625.
    Entry B: dz2_0 = 0.5, dz1 = (0.5, 0).  Weight gradients take the rounded dz,
    bias gradients the unrounded ones; in fp64 mode nothing is rounded."""
    W1 = np.zeros((fsai.N_HID, fsai.N_IN)); b1 = np.zeros(fsai.N_HID)
    W2 = np.zeros((fsai.N_HID, fsai.N_HID)); b2 = np.zeros(fsai.N_HID)
    W3 = np.zeros(fsai.N_HID)
    dz2a = 0.50390625 if rounded else 0.5029296875       # weight-gradient input of entry A
    dz1a = (0.50390625, 1.515625) if rounded else (0.5029296875, 1.5087890625)
    W3[0] = 3.5 * D_A + 2.75                 # h2_0 dout summed over A and B
    b3 = D_A + 1.0
    W2[0, 0] = 3.0 * dz2a + 3.0 * 0.5        # dz2_0 h1_0
    W2[0, 1] = 0.25 * dz2a                   # h1_1 = 0.25 in A, 0 in B
    b2[0] = 0.5029296875 + 0.5
    W1[0, 0], W1[1, 0] = 7.0 * dz1a[0], 7.0 * dz1a[1]
    W1[0, 3] = 1.5 * dz1a[0] + 1.5 * 0.5
    W1[0, 7] = 0.25 * dz1a[0] + 1.0 * 0.5
    W1[1, 3], W1[1, 7] = 1.5 * dz1a[1], 0.25 * dz1a[1]
    b1[0] = 0.50390625 + 0.5 if rounded else 0.5029296875 + 0.5
    b1[1] = 1.51171875 if rounded else 1.5087890625
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, [b3]])


def backward_pin_holds(backward):
    p = hand_network()
    F, dout = hand_backward_case()
    for rnd in (True, False):
        o, cache = fsai.mlp_forward(p, F, round_bf16=rnd)
        if not np.array_equal(o, [0.5 * 3.5 + 0.125, 0.5 * 2.75 + 0.125]):
            return False
        if not np.array_equal(backward(dout, cache), hand_backward_expected(rnd)):
            return False
    return True


def test_mlp_backward_by_hand():
    """F7 on a network evaluated by hand, in both precision modes: where dz2 and dz1 are
    rounded to bf16 (before the weight-gradient products and before dh1 = dz2 W2), that
    the bias gradients take the unrounded values, the ReLU masks of both layers and the
    orientation of W2 in dh1."""
    assert backward_pin_holds(fsai.mlp_backward)


# Plausible mistakes in the backward pass, each planted in a copy of mlp_backward.
# Moving a rounding to after a ReLU mask is not among them: the mask is 0 or 1, so the
# two orders give the same bits.
BACKWARD_MUTANTS = {
    "dz1 from the unrounded dz2": ("dz1 = (dz2r @ W2)", "dz1 = (dz2 @ W2)"),
    "dW2 from the unrounded dz2": ("dW2 = dz2r.T @ h1", "dW2 = dz2.T @ h1"),
    "dW1 from the unrounded dz1": ("dW1 = dz1r.T @ X", "dW1 = dz1.T @ X"),
    "db2 from the rounded dz2": ("db2 = dz2.sum(0)", "db2 = dz2r.sum(0)"),
    "db1 from the rounded dz1": ("db1 = dz1.sum(0)", "db1 = dz1r.sum(0)"),
    "W2 transposed in dh1": ("(dz2r @ W2)", "(dz2r @ W2.T)"),
    "first-layer ReLU mask dropped": ("* (z1 > 0)", "* 1.0"),
    "second-layer ReLU mask dropped": ("* (z2 > 0)", "* 1.0"),
    "dz2 not rounded": ("dz2r = rnd(dz2)", "dz2r = dz2"),
}


@pytest.mark.parametrize("name", sorted(BACKWARD_MUTANTS))
def test_backward_pin_catches_planted_mistakes(name):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fsai.mlp_backward))
    old, new = BACKWARD_MUTANTS[name]
    assert src.count(old) == 1, (name, old)
    ns = dict(vars(fsai))
    exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)
    assert not backward_pin_holds(ns["mlp_backward"]), name
