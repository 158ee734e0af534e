"""Symbolic Cholesky of a sparse symmetric pattern: oracle form.

TEST INFRASTRUCTURE (see the package docstring).  Plain numpy on dense boolean matrices,
for small cases only.

Algorithm 2 keeps Lambda sparse, and its line search needs log det of Lambda + alpha D
(Section 4; Section 2.3 computes log det from a Cholesky factor).  For a sparse Lambda that
factor is a sparse Cholesky, whose structure depends only on the pattern and the pivot
order.  The definition used here is the elimination game: with the pattern permuted to
the pivot order, eliminating pivot k joins every pair of rows r, s > k that have an entry
in column k; the pattern of L is the lower triangle at the end.  From it:

  * the elimination tree: parent(k) = min { r > k : L_rk != 0 }, or -1;
  * column counts: the entries of column k of L, the diagonal included;
  * fill: entries of L that were not in the lower triangle of the permuted pattern.
"""
from __future__ import annotations

import numpy as np


def pattern_from_csr(q, row_ptr, col) -> np.ndarray:
    """Dense boolean symmetric pattern with a full diagonal from CSR entries (either or
    both triangles given)."""
    A = np.zeros((q, q), dtype=bool)
    row_ptr = np.asarray(row_ptr)
    col = np.asarray(col)
    for i in range(q):
        for t in range(row_ptr[i], row_ptr[i + 1]):
            A[i, col[t]] = True
            A[col[t], i] = True
    np.fill_diagonal(A, True)
    return A


def cholesky_pattern(A: np.ndarray, perm) -> np.ndarray:
    """Pattern of L for the pivot order perm (perm[k] = original index of pivot k), by
    the elimination game."""
    perm = np.asarray(perm)
    B = A[np.ix_(perm, perm)].copy()
    q = B.shape[0]
    for k in range(q):
        rows = np.flatnonzero(B[k + 1:, k]) + k + 1
        if rows.size:
            B[np.ix_(rows, rows)] = True
    return np.tril(B)


def etree(L: np.ndarray) -> np.ndarray:
    """parent(k) = the first row below the diagonal with an entry in column k, or -1."""
    q = L.shape[0]
    parent = np.full(q, -1, dtype=np.int64)
    for k in range(q):
        below = np.flatnonzero(L[k + 1:, k])
        if below.size:
            parent[k] = k + 1 + below[0]
    return parent


def column_counts(L: np.ndarray) -> np.ndarray:
    return L.sum(axis=0).astype(np.int64)


def analyse(q, row_ptr, col, perm):
    """(parent, colcount, nnz_L, fill) for the pivot order perm."""
    A = pattern_from_csr(q, row_ptr, col)
    L = cholesky_pattern(A, perm)
    cc = column_counts(L)
    perm = np.asarray(perm)
    fill = int(L.sum()) - int(np.tril(A[np.ix_(perm, perm)]).sum())
    return etree(L), cc, int(cc.sum()), fill


def fundamental_supernodes(L: np.ndarray) -> np.ndarray:
    """Start columns of the fundamental supernodes of the factor pattern L (with q as a
    final sentinel): column k + 1 continues the supernode of column k when the pattern of
    column k below its diagonal is exactly the pattern of column k + 1 (diagonal included),
    and k is the only child of k + 1 in the elimination tree."""
    q = L.shape[0]
    parent = etree(L)
    children = np.bincount(parent[parent >= 0], minlength=q) if q else np.zeros(0, int)
    starts = [0] if q else []
    for k in range(q - 1):
        same = np.array_equal(L[k + 1:, k], L[k + 1:, k + 1])
        if not (same and children[k + 1] == 1):
            starts.append(k + 1)
    return np.array(starts + [q], dtype=np.int64)


def minimum_degree_order(A: np.ndarray, dense_rest: float = 0.9) -> np.ndarray:
    """Minimum-degree pivot order by the elimination game on the pattern A (dense boolean,
    symmetric): repeatedly take the remaining vertex of least degree in the elimination
    graph (ties: lower index), join its neighbours into a clique and remove it.  Once more
    than 64 vertices remain and the least degree plus one reaches ``dense_rest`` times their
    number, the remaining graph is nearly complete and the rest follow in (degree, index)
    order."""
    q = A.shape[0]
    G = A.copy()
    np.fill_diagonal(G, False)
    alive = np.ones(q, dtype=bool)
    order = []
    while len(order) < q:
        idx = np.flatnonzero(alive)
        deg = G[np.ix_(idx, idx)].sum(axis=1)
        remaining = idx.size
        best = int(np.lexsort((idx, deg))[0])
        if remaining > 64 and deg[best] + 1 >= dense_rest * remaining:
            rest = idx[np.lexsort((idx, deg))]
            order.extend(int(v) for v in rest)
            break
        v = int(idx[best])
        nb = np.flatnonzero(G[v] & alive)
        G[np.ix_(nb, nb)] = True
        G[nb, nb] = False
        alive[v] = False
        G[v, :] = False
        G[:, v] = False
        order.append(v)
    return np.array(order, dtype=np.int64)


def numeric_factor(A: np.ndarray, perm):
    """The numeric factor the sparse Cholesky computes, by its definition: L lower
    triangular with a positive diagonal and L L^T = P A P^T (A symmetric positive definite,
    dense; perm[k] = original index of pivot k), which fixes L uniquely.  Returns
    (L, log det A) with log det A = 2 sum_k log L_kk (Section 2.3 takes log det from the
    factor).  LAPACK's dense Cholesky is the library step."""
    perm = np.asarray(perm)
    L = np.linalg.cholesky(A[np.ix_(perm, perm)])
    return L, 2.0 * float(np.sum(np.log(np.diag(L))))
