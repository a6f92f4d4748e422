"""Shared test helpers: device copies of generated CSR matrices and adversarial
row-length patterns.  Holds no CG arithmetic."""
import numpy as np

import cgproblems as gen


def to_device(A):
    import torch
    return (torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.colind).cuda(),
            torch.from_numpy(A.vals).cuda())


def adversarial(n, seed, long_rows=(), empty_every=0, max_len=12):
    """Random symmetric-pattern-free CSR with chosen row lengths: short random rows,
    some empty rows and a few very long rows (dense-ish), sorted columns per row."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, max_len + 1, size=n)
    if empty_every:
        lens[::empty_every] = 0
    for r, L in long_rows:
        lens[r] = L
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum(lens)
    colind = np.empty(rowptr[-1], dtype=np.int32)
    for i in range(n):
        L = lens[i]
        if L:
            colind[rowptr[i]:rowptr[i + 1]] = np.sort(rng.choice(n, size=min(L, n), replace=False))
    vals = rng.uniform(-1.0, 1.0, size=rowptr[-1])
    return gen.CSR(n, rowptr.astype(np.int32), colind, vals, f"adversarial_n{n}_s{seed}")


def spd_from_pattern(n, seed, long_rows=(), max_len=8):
    """SPD matrix with an uneven row-length mix: symmetric random couplings (including a
    few dense rows) made strictly diagonally dominant."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        k = rng.integers(0, max_len)
        js = rng.integers(0, n, size=k)
        rows += [i] * k
        cols += list(js)
    for r, L in long_rows:
        js = rng.choice(n, size=min(L, n), replace=False)
        rows += [r] * len(js)
        cols += list(js)
    M = sp.coo_matrix((rng.uniform(-1, 0, len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    M = M + M.T
    M.setdiag(0)
    M.eliminate_zeros()
    d = np.asarray(abs(M).sum(axis=1)).ravel() + rng.uniform(0.1, 1.0, n)
    M = (M + sp.diags(d)).tocsr()
    M.sort_indices()
    return gen.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                   M.data.astype(np.float64), f"spd_pattern_n{n}_s{seed}")


def random_graph_spd(n, seed, matchings=2):
    """SPD graph Laplacian + I of the union of `matchings` random perfect matchings:
    every row has at most 2*matchings off-diagonal entries at random columns, so the
    loop matrix takes the uniform-width slice layout without the diagonal layout."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for _ in range(matchings):
        perm = rng.permutation(n)
        a, b = perm[0::2], perm[1::2]
        rows += list(a) + list(b)
        cols += list(b) + list(a)
    W = sp.coo_matrix((rng.uniform(0.5, 1.5, len(rows)), (rows, cols)), shape=(n, n)).tocsr()
    W = (W + W.T) * 0.5
    W.setdiag(0)
    W.eliminate_zeros()
    d = np.asarray(W.sum(axis=1)).ravel() + 1.0
    M = (sp.diags(d) - W).tocsr()
    M.sort_indices()
    return gen.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32),
                   M.data.astype(np.float64), f"graph_spd_n{n}_s{seed}")


def hub_graph_spd(n, seed, hub_len):
    """A power-law graph Laplacian (cgproblems.graph_spd, the CSR loop layout's input
    class) plus the Laplacian of a star joining row 0 to hub_len random rows (weight 0.5):
    still SPD, with one row longer than a row block's 2044-entry cap."""
    import scipy.sparse as sp
    import cgproblems as gen
    A = gen.graph_spd(n, 600, seed).to_scipy().tocoo()
    rng = np.random.default_rng(seed)
    leaves = rng.choice(np.arange(1, n), size=hub_len, replace=False)
    w = 0.5
    r = np.concatenate([np.zeros(hub_len, np.int64), leaves, [0], leaves])
    c = np.concatenate([leaves, np.zeros(hub_len, np.int64), [0], leaves])
    v = np.concatenate([np.full(2 * hub_len, -w), [w * hub_len], np.full(hub_len, w)])
    M = (A + sp.coo_matrix((v, (r, c)), shape=(n, n))).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return gen.CSR(n, M.indptr.astype(np.int32), M.indices.astype(np.int32), M.data.astype(np.float64),
                   f"hub_graph_n{n}_s{seed}_h{hub_len}")
