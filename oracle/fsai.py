"""Learned FSAI preconditioner oracle -- TEST INFRASTRUCTURE ONLY.

Plain numpy (fp64) restatement of the factorized sparse approximate inverse
preconditioner M^-1 = G^T G that the CUDA library builds, either classically
(Kolotilina & Yeremin, 1993) or from a small MLP, and of the MLP's training
loss and gradients.  Only the test suite, the smoke check and the benchmark's
CPU legs may use it; it shares nothing with the CUDA path but the generated
inputs.  The paper has no preconditioner beyond its plain CG (Alg. 1); every
definition here is a project reading, listed as F1-F8:

  F1 pattern: G is lower triangular with the pattern of tril(A) (the CSR of A
     must have strictly increasing columns in each row and a positive diagonal).
  F2 classic FSAI: row i solves A[P_i, P_i] y = e_i on its pattern P_i and sets
     g_i = y / sqrt(y_i); then (G A G^T)_ii = 1 and G minimises the Kaporin
     number over the pattern (Kolotilina & Yeremin 1993; Kaporin 1994).
  F3 features of an entry (i, j) of tril(A), d = diag(A), s(i,k) = A_ik / sqrt(d_i d_k):
     [0:8]   one-hot slot of j - i among the sorted non-positive offsets of A,
     [8]     s(i, j),
     [9]     log(d_j / d_i),
     [10:19] s(i, i + o_m) for the sorted distinct offsets o_m of A (0 if absent),
     [19:28] s(j, j + o_m) likewise,
     [28]    1, [29:32] 0.
     A has at most 9 distinct offsets (j - i) over all entries.
  F4 MLP 32 -> 64 -> 64 -> 1, ReLU; parameters in one fp32 vector
     [W1 (64x32, row = output) | b1 | W2 (64x64) | b2 | W3 (64) | b3].
     Kernel precision points (the bf16 flag): parameters and features rounded to
     bf16 (round to nearest even), layer sums in fp32 or better, h1 = bf16(relu(z1)),
     h2 = relu(z2) unrounded, o = W3 . h2 + b3.
  F5 G from the output o of each entry: G_ij = o / sqrt(d_j) (j < i),
     G_ii = softplus(o + c0) / sqrt(d_i) with softplus(c0) = 1, so o = 0 gives
     G = D^-1/2 (Jacobi) and G_ii > 0 makes G^T G SPD.
  F6 loss = Kaporin term + lam * residual term:
     L_K = log((1/n) sum_i g_i^T A g_i) - (2/n) sum_i log G_ii   (Kaporin 1994,
           log of the K-condition number of G A G^T up to a constant),
     L_R = mean_k ||A G^T G r_k - r_k||^2 / ||r_k||^2 over stored residuals r_k.
  F7 backward (kernel precision points): dz2 and dz1 rounded to bf16 as the
     inputs of the weight-gradient and dh1 products; bias gradients from the
     unrounded values.
  F8 Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _Result, _csr, _load, _p, Solve

N_IN, N_HID = 32, 64
N_PARAMS = N_HID * N_IN + N_HID + N_HID * N_HID + N_HID + N_HID + 1
C0 = math.log(math.e - 1.0)  # softplus(C0) = 1
MAX_OFFSETS = 9
TRIL_SLOTS = 8


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits, ties to even), returned
    as fp64; exact for every finite input in bf16's normal range."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)               # x = m 2^e, |m| in [0.5, 1)
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    assert p.size == N_PARAMS
    o = 0
    W1 = p[o:o + N_HID * N_IN].reshape(N_HID, N_IN); o += N_HID * N_IN
    b1 = p[o:o + N_HID]; o += N_HID
    W2 = p[o:o + N_HID * N_HID].reshape(N_HID, N_HID); o += N_HID * N_HID
    b2 = p[o:o + N_HID]; o += N_HID
    W3 = p[o:o + N_HID]; o += N_HID
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, W3, [b3]])


def init_params(seed: int) -> np.ndarray:
    """He-normal hidden layers, zero biases, zero output layer (so G = D^-1/2 at start)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / N_IN), (N_HID, N_IN))
    W2 = rng.normal(0.0, math.sqrt(2.0 / N_HID), (N_HID, N_HID))
    z = np.zeros(N_HID)
    return pack(W1, z, W2, z, np.zeros(N_HID), 0.0).astype(np.float32)


# ------------------------------------------------------------------ pattern (F1)

def _rows(A):
    return np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.rowptr.astype(np.int64)))


def diag(A) -> np.ndarray:
    rows = _rows(A)
    d = np.zeros(A.n)
    m = A.colind == rows
    np.add.at(d, rows[m], A.vals[m])
    return d


def check_matrix(A):
    rows = _rows(A)
    ci = A.colind.astype(np.int64)
    same_row = rows[1:] == rows[:-1]
    if np.any(ci[1:][same_row] <= ci[:-1][same_row]):
        raise ValueError("columns must increase strictly within each row")
    d = diag(A)
    if np.any(~(d > 0)):
        raise ValueError("FSAI needs a positive diagonal")
    return d


def tril(A):
    """Entries of tril(A) in CSR order: (rowptr, col, source index into A's arrays)."""
    rows = _rows(A)
    keep = A.colind <= rows
    src = np.nonzero(keep)[0]
    cnt = np.bincount(rows[keep], minlength=A.n)
    trp = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    return trp, A.colind[src].astype(np.int32), src


def g_matrix(A, gvals):
    """G as a scipy CSR matrix from its values in tril(A) order."""
    import scipy.sparse as sp
    trp, tci, _ = tril(A)
    return sp.csr_matrix((np.asarray(gvals, dtype=np.float64), tci, trp), shape=(A.n, A.n))


# ------------------------------------------------------------------ classic FSAI (F2)

def classic(A) -> np.ndarray:
    """Classic FSAI values in tril(A) order: per row, a small dense SPD solve."""
    check_matrix(A)
    trp, tci, _ = tril(A)
    S = A.to_scipy().tocsr()
    g = np.empty(len(tci))
    for i in range(A.n):
        P = tci[trp[i]:trp[i + 1]]
        loc = S[P][:, P].toarray()
        e = np.zeros(len(P))
        e[-1] = 1.0                  # P is ascending and ends with i
        y = np.linalg.solve(loc, e)
        if not y[-1] > 0:
            raise ValueError(f"row {i}: local matrix is not SPD")
        g[trp[i]:trp[i + 1]] = y / math.sqrt(y[-1])
    return g


# ------------------------------------------------------------------ features (F3)

def offsets(A) -> np.ndarray:
    offs = np.unique(A.colind.astype(np.int64) - _rows(A))
    if len(offs) > MAX_OFFSETS:
        raise ValueError(f"{len(offs)} distinct offsets (the features take at most {MAX_OFFSETS})")
    return offs


def features(A) -> np.ndarray:
    """F3 feature rows (fp64) of the entries of tril(A), in tril(A) order."""
    d = check_matrix(A)
    rows = _rows(A)
    ci = A.colind.astype(np.int64)
    offs = offsets(A)
    slot = np.searchsorted(offs, ci - rows)
    s_all = A.vals / np.sqrt(d[rows] * d[ci])
    R = np.zeros((A.n, MAX_OFFSETS))
    R[rows, slot] = s_all
    tslots = offs[offs <= 0]
    _, tci, src = tril(A)
    i = rows[src]
    j = ci[src]
    F = np.zeros((len(src), N_IN))
    F[np.arange(len(src)), np.searchsorted(tslots, j - i)] = 1.0
    F[:, 8] = s_all[src]
    F[:, 9] = np.log(d[j] / d[i])
    F[:, 10:19] = R[i]
    F[:, 19:28] = R[j]
    F[:, 28] = 1.0
    return F


# ------------------------------------------------------------------ MLP (F4, F7)

def mlp_forward(params, F, round_bf16=True):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    rnd = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = (rnd(v) for v in (W1, b1, W2, b2, W3, b3))
    X = rnd(F)
    z1 = X @ W1.T + b1
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W3 + b3
    return o, (X, z1, h1, z2, h2, W2, W3, rnd)


def mlp_backward(dout, cache):
    """Gradient of sum(dout * o) with respect to the parameter vector."""
    X, z1, h1, z2, h2, W2, W3, rnd = cache
    dW3 = h2.T @ dout
    db3 = dout.sum()
    dz2 = np.outer(dout, W3) * (z2 > 0)
    dz2r = rnd(dz2)
    dW2 = dz2r.T @ h1
    db2 = dz2.sum(0)
    dz1 = (dz2r @ W2) * (z1 > 0)
    dz1r = rnd(dz1)
    dW1 = dz1r.T @ X
    db1 = dz1.sum(0)
    return pack(dW1, db1, dW2, db2, dW3, db3)


# ------------------------------------------------------------------ G from the output (F5)

def _softplus(x):
    return np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))), np.log1p(np.exp(x)))


def _sigmoid(x):
    return np.where(x >= 0, 1.0 / (1.0 + np.exp(-np.abs(x))), np.exp(x) / (1.0 + np.exp(x)))


def g_from_output(A, o):
    """G values (tril(A) order) and dG/do from the MLP outputs o."""
    d = diag(A)
    rows = _rows(A)
    _, tci, src = tril(A)
    i = rows[src]
    j = tci.astype(np.int64)
    on = i == j
    g = np.where(on, _softplus(o + C0) / np.sqrt(d[i]), o / np.sqrt(d[j]))
    dg = np.where(on, _sigmoid(o + C0) / np.sqrt(d[i]), 1.0 / np.sqrt(d[j]))
    return g, dg


def learned(A, params, round_bf16=True):
    o, _ = mlp_forward(params, features(A), round_bf16)
    return g_from_output(A, o)[0]


# ------------------------------------------------------------------ loss (F6)

def kaporin(A, gvals):
    """L_K and dL_K/dG (tril(A) order)."""
    G = g_matrix(A, gvals)
    S_A = A.to_scipy().tocsr()
    GA = (G @ S_A).tocsr()
    quad = np.asarray(GA.multiply(G).sum(axis=1)).ravel()   # g_i^T A g_i
    n = A.n
    S = quad.mean()
    gd = G.diagonal()
    L = math.log(S) - 2.0 / n * np.sum(np.log(gd))
    trp, tci, _ = tril(A)
    rows = np.repeat(np.arange(n), np.diff(trp))
    grad = 2.0 / (n * S) * np.asarray(GA[rows, tci]).ravel()
    on = rows == tci
    grad[on] -= 2.0 / (n * gd[rows[on]])
    return L, grad


def residual_term(A, gvals, R):
    """L_R and dL_R/dG for residual vectors R (k x n)."""
    G = g_matrix(A, gvals)
    S_A = A.to_scipy().tocsr()
    trp, tci, _ = tril(A)
    rows = np.repeat(np.arange(A.n), np.diff(trp))
    L = 0.0
    grad = np.zeros(len(tci))
    for r in np.atleast_2d(R):
        rn2 = float(r @ r)
        u = G @ r
        e = S_A @ (G.T @ u) - r
        Ae = S_A @ e
        GAe = G @ Ae
        L += float(e @ e) / rn2
        grad += 2.0 / rn2 * (u[rows] * Ae[tci] + GAe[rows] * r[tci])
    k = len(np.atleast_2d(R))
    return L / k, grad / k


def loss_and_grad(A, params, R=None, lam=0.1, round_bf16=True):
    """Total loss and its gradient with respect to the parameter vector."""
    F = features(A)
    o, cache = mlp_forward(params, F, round_bf16)
    g, dgdo = g_from_output(A, o)
    L, dG = kaporin(A, g)
    if R is not None and len(R):
        LR, dR = residual_term(A, g, R)
        L += lam * LR
        dG = dG + lam * dR
    return L, mlp_backward(dG * dgdo, cache)


def adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (F8); returns new (params, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


# ------------------------------------------------------------------ PCG with G^T G (oracle.c, R7)

def _bind_fsai(lib):
    if getattr(lib, "_fsai_bound", False):
        return lib
    P, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.or_pcg_fsai.argtypes = [i64, P, P, P, P, P, P, P, P, f64, i32, i32, P, P,
                                ctypes.POINTER(_Result)]
    lib.or_pcg_fsai.restype = ctypes.c_int
    lib.or_pcg_ir_fsai.argtypes = [i64, P, P, P, P, P, P, P, P, f64, f64, i32, i32, P,
                                   ctypes.POINTER(_Result)]
    lib.or_pcg_ir_fsai.restype = ctypes.c_int
    lib.or_pcg_ru_fsai.argtypes = lib.or_pcg_ir_fsai.argtypes
    lib.or_pcg_ru_fsai.restype = ctypes.c_int
    lib._fsai_bound = True
    return lib


def pcg(A, gvals, b, x0=None, tol=1e-8, maxit=1000, max_restarts=3, res_hist=False):
    """PCG with M^-1 = G^T G (R7), G given by its values in tril(A) order.  The
    returned Solve carries rz_min (smallest r.z seen) as an extra attribute."""
    lib = _bind_fsai(_load())
    n, rp, ci, va = _csr(A)
    trp, tci, _ = tril(A)
    gv = np.ascontiguousarray(gvals, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rh = np.full(maxit + 1, np.nan) if res_hist else None
    rz = ctypes.c_double(0.0)
    res = _Result()
    lib.or_pcg_fsai(n, _p(rp), _p(ci), _p(va), _p(trp), _p(tci), _p(gv), _p(b), _p(x), tol, maxit,
                    max_restarts, _p(rh), ctypes.byref(rz), ctypes.byref(res))
    s = Solve(x, res.status, res.iters, res.restarts, res.relres_rec, res.relres_true,
              None if rh is None else rh[: res.iters + 1])
    s.rz_min = rz.value
    return s


def pcg_ir(A, gvals, b, x0=None, tol=1e-8, tol_in=1e-4, maxit=100000, max_outer=30,
           carry=False) -> Solve:
    """fp32-inner / fp64-outer refinement (R6) with the inner M^-1 = G32^T G32 (R7);
    carry=True carries the search direction over the fp64 updates (R8)."""
    lib = _bind_fsai(_load())
    n, rp, ci, va = _csr(A)
    trp, tci, _ = tril(A)
    gv = np.ascontiguousarray(gvals, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    oh = np.full(max_outer + 1, np.nan)
    res = _Result()
    fn = lib.or_pcg_ru_fsai if carry else lib.or_pcg_ir_fsai
    fn(n, _p(rp), _p(ci), _p(va), _p(trp), _p(tci), _p(gv), _p(b), _p(x), tol, tol_in, maxit,
       max_outer, _p(oh), ctypes.byref(res))
    return Solve(x, res.status, res.iters, res.restarts, res.relres_rec, res.relres_true,
                 outer_hist=oh[: res.restarts + 1])
