"""Pins of the oracle's symbolic Cholesky (CPU): the elimination game's pattern equals the
nonzero pattern of a numeric Cholesky factor (LAPACK through numpy) of a matrix with that
sparsity and generic values, and closed forms on a path, an arrow and a dense pattern."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import symbolic


def csr_of(A):
    m = sp.csr_matrix(A)
    return m.indptr, m.indices


def random_pattern(q, m, seed):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, q, m)
    j = rng.integers(0, q, m)
    A = np.zeros((q, q), dtype=bool)
    A[i, j] = True
    A[j, i] = True
    np.fill_diagonal(A, True)
    return A


@pytest.mark.parametrize("q,m,seed", [(30, 40, 1), (60, 90, 2), (45, 300, 3), (1, 0, 4)])
def test_pattern_equals_numeric_cholesky(q, m, seed):
    """Generic values on the pattern, made diagonally dominant: every structurally nonzero
    entry of L is nonzero, and every structural zero is computed as an exact zero."""
    rng = np.random.default_rng(seed + 100)
    A = random_pattern(q, m, seed)
    V = np.where(A, rng.uniform(0.1, 1.0, (q, q)), 0.0)
    V = np.triu(V, 1)
    V = V + V.T
    V += np.diag(np.abs(V).sum(axis=1) + 1.0)
    for perm in (np.arange(q), rng.permutation(q)):
        Lnum = np.linalg.cholesky(V[np.ix_(perm, perm)])
        rp, ci = csr_of(A)
        L = symbolic.cholesky_pattern(symbolic.pattern_from_csr(q, rp, ci), perm)
        assert np.array_equal(L, Lnum != 0.0)


def test_path_has_no_fill():
    q = 10
    A = np.eye(q, dtype=bool) | np.eye(q, k=1, dtype=bool) | np.eye(q, k=-1, dtype=bool)
    rp, ci = csr_of(A)
    parent, cc, nnz, fill = symbolic.analyse(q, rp, ci, np.arange(q))
    assert parent.tolist() == list(range(1, q)) + [-1]
    assert cc.tolist() == [2] * (q - 1) + [1]
    assert nnz == 2 * q - 1 and fill == 0


def test_arrow_order_decides_fill():
    """A hub joined to every other column: eliminated first it fills the whole factor,
    eliminated last it fills nothing."""
    q = 8
    A = np.eye(q, dtype=bool)
    A[0, :] = A[:, 0] = True
    rp, ci = csr_of(A)
    _, cc, nnz, fill = symbolic.analyse(q, rp, ci, np.arange(q))
    assert nnz == q * (q + 1) // 2 and fill == (q - 1) * (q - 2) // 2
    hub_last = np.r_[np.arange(1, q), 0]
    parent, cc, nnz, fill = symbolic.analyse(q, rp, ci, hub_last)
    assert nnz == 2 * q - 1 and fill == 0
    assert parent.tolist() == [q - 1] * (q - 1) + [-1]


def test_dense_pattern():
    q = 6
    A = np.ones((q, q), dtype=bool)
    rp, ci = csr_of(A)
    parent, cc, nnz, fill = symbolic.analyse(q, rp, ci, np.arange(q))
    assert cc.tolist() == list(range(q, 0, -1)) and fill == 0
    assert parent.tolist() == list(range(1, q)) + [-1]


def test_supernodes_closed_forms():
    """A dense pattern is one supernode; a path splits into single columns except its last
    two (column q-2 below its diagonal is {q-1}, the pattern of the last column); with a
    hub eliminated last every column stands alone (the hub has q-1 children)."""
    q = 6
    L = symbolic.cholesky_pattern(np.ones((q, q), dtype=bool), np.arange(q))
    assert symbolic.fundamental_supernodes(L).tolist() == [0, q]
    A = np.eye(q, dtype=bool) | np.eye(q, k=1, dtype=bool) | np.eye(q, k=-1, dtype=bool)
    L = symbolic.cholesky_pattern(A, np.arange(q))
    assert symbolic.fundamental_supernodes(L).tolist() == [0, 1, 2, 3, 4, q]
    H = np.eye(q, dtype=bool)
    H[0, :] = H[:, 0] = True
    L = symbolic.cholesky_pattern(H, np.r_[np.arange(1, q), 0])
    assert symbolic.fundamental_supernodes(L).tolist() == list(range(q)) + [q]


def test_supernode_columns_share_their_pattern():
    """Within every supernode each column's pattern below the diagonal is the next
    column's pattern: the columns form one dense block with a common row set."""
    A = random_pattern(50, 120, 9)
    L = symbolic.cholesky_pattern(A, np.arange(50))
    s = symbolic.fundamental_supernodes(L)
    assert s[0] == 0 and s[-1] == 50 and np.all(np.diff(s) > 0)
    for a, b in zip(s[:-1], s[1:]):
        for k in range(a, b - 1):
            assert np.array_equal(L[k + 1:, k], L[k + 1:, k + 1])


def test_minimum_degree_closed_forms():
    """On a forest every step takes a vertex of degree at most one (no fill); a star's
    leaves go first, the hub once it is down to one leaf (the tie goes to its lower index);
    a complete graph is taken in index order; a path from an end."""
    q = 7
    star = np.eye(q, dtype=bool)
    star[3, :] = star[:, 3] = True
    assert symbolic.minimum_degree_order(star).tolist() == [0, 1, 2, 4, 5, 3, 6]
    assert symbolic.minimum_degree_order(np.ones((q, q), dtype=bool)).tolist() == list(range(q))
    A = np.eye(q, dtype=bool) | np.eye(q, k=1, dtype=bool) | np.eye(q, k=-1, dtype=bool)
    assert symbolic.minimum_degree_order(A).tolist() == list(range(q))
    rng = np.random.default_rng(3)
    q = 60
    F = np.eye(q, dtype=bool)
    for v in range(1, q):
        if v % 7:
            u = rng.integers(0, v)
            F[u, v] = F[v, u] = True
    L = symbolic.cholesky_pattern(F, symbolic.minimum_degree_order(F))
    assert L.sum() == q + (F.sum() - q) // 2            # no fill


def test_minimum_degree_dense_rest():
    """More than 64 vertices left, least degree + 1 >= 0.9 x remaining: the rest in (degree,
    index) order, which on a complete graph is the index order from the first step."""
    q = 80
    A = np.ones((q, q), dtype=bool)
    A[0, 1] = A[1, 0] = False                           # degrees 78, 78, then 79 ...
    order = symbolic.minimum_degree_order(A)
    assert order.tolist() == list(range(q))


# ---- the numeric factor (oracle.symbolic.numeric_factor) ----

def second_difference(q):
    """T_q: 2 on the diagonal, -1 beside it; det T_q = q + 1."""
    return 2.0 * np.eye(q) - np.eye(q, k=1) - np.eye(q, k=-1)


@pytest.mark.parametrize("q", [1, 2, 7, 50])
def test_numeric_factor_second_difference_closed_form(q):
    L, ld = symbolic.numeric_factor(second_difference(q), np.arange(q))
    k = np.arange(q)
    # the recurrence d_k = 2 - 1 / d_{k-1}, d_0 = 2, gives d_k = (k + 2) / (k + 1)
    np.testing.assert_allclose(np.diag(L), np.sqrt((k + 2) / (k + 1)), rtol=1e-14)
    np.testing.assert_allclose(np.diag(L, -1), -np.sqrt((k[:-1] + 1) / (k[:-1] + 2)),
                               rtol=1e-14)
    assert abs(ld - np.log(q + 1)) <= 1e-13 * max(1.0, np.log(q + 1))


def test_numeric_factor_any_pivot_order_same_determinant():
    q = 40
    rng = np.random.default_rng(5)
    perm = rng.permutation(q)
    A = second_difference(q)
    L, ld = symbolic.numeric_factor(A, perm)
    assert abs(ld - np.log(q + 1)) <= 1e-12
    np.testing.assert_allclose(L @ L.T, A[np.ix_(perm, perm)], atol=1e-13)
    assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)


def test_numeric_factor_against_lu_determinant():
    import scipy.linalg as sla
    import synth
    rng = np.random.default_rng(11)
    q = 80
    A = synth.random_sparse_precision(q, 4.0, rng, base=synth.chain_precision(q)).toarray()
    perm = rng.permutation(q)
    L, ld = symbolic.numeric_factor(A, perm)
    lu, piv = sla.lu_factor(A)  # a different factorisation of the same matrix
    sign = np.prod(np.sign(np.diag(lu))) * (-1) ** np.count_nonzero(piv != np.arange(q))
    assert sign > 0
    assert abs(ld - np.sum(np.log(np.abs(np.diag(lu))))) <= 1e-11 * abs(ld)
    np.testing.assert_allclose(L @ L.T, A[np.ix_(perm, perm)], atol=1e-12)
    # its nonzeros lie inside the elimination game's pattern for the same order
    P = symbolic.cholesky_pattern(A != 0, perm)
    assert not np.any((np.abs(L) > 0) & ~P)
