"""Symbolic sparse Cholesky (cggm_chol_symbolic, host code of the library; no GPU) against
the oracle's elimination game.  Integer work, so bit-exact: for caller-given pivot orders
the elimination tree, the column counts and nnz(L) equal the oracle's.  The orders the
library computes are checked by what they must achieve: valid permutations; no fill on a
relabelled path (reverse Cuthill-McKee, minimum degree) or forest (minimum degree); fill
inside the band of a relabelled banded pattern (reverse Cuthill-McKee); far less fill than
the other orders on a chain with random links (minimum degree)."""
import time

import numpy as np
import pytest
import scipy.sparse as sp

import paper_1509_04681_gb300 as cg
from oracle import symbolic


def random_csr(q, m, seed, upper_only=False):
    rng = np.random.default_rng(seed)
    i = rng.integers(0, q, m)
    j = rng.integers(0, q, m)
    if upper_only:
        i, j = np.minimum(i, j), np.maximum(i, j)
    A = sp.csr_matrix((np.ones(m), (i, j)), shape=(q, q))
    A.sum_duplicates()
    return A.indptr, A.indices


@pytest.mark.parametrize("q,m,seed", [(1, 0, 1), (12, 10, 2), (40, 60, 3), (80, 160, 4),
                                      (120, 130, 5), (60, 900, 6)])
def test_given_orders_match_the_oracle(q, m, seed):
    rp, ci = random_csr(q, m, seed)
    rng = np.random.default_rng(seed)
    for perm in (np.arange(q), rng.permutation(q), rng.permutation(q)[::-1].copy()):
        p_out, parent, cc, nnz = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_GIVEN, perm)
        r_parent, r_cc, r_nnz, _ = symbolic.analyse(q, rp, ci, perm)
        assert np.array_equal(p_out, perm)
        assert np.array_equal(parent, r_parent)
        assert np.array_equal(cc, r_cc)
        assert nnz == r_nnz
    # the natural order is the identity permutation
    _, parent, cc, nnz = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_NATURAL)
    r_parent, r_cc, r_nnz, _ = symbolic.analyse(q, rp, ci, np.arange(q))
    assert np.array_equal(parent, r_parent) and np.array_equal(cc, r_cc) and nnz == r_nnz


def test_one_triangle_is_enough():
    q = 50
    rp_u, ci_u = random_csr(q, 120, 7, upper_only=True)
    U = sp.csr_matrix((np.ones(len(ci_u)), ci_u, rp_u), shape=(q, q))
    F = (U + U.T).tocsr()
    a = cg.chol_symbolic(q, rp_u, ci_u, cg.CGGM_ORDER_NATURAL)
    b = cg.chol_symbolic(q, F.indptr, F.indices, cg.CGGM_ORDER_NATURAL)
    assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3])) and a[3] == b[3]


def relabelled(A, seed):
    q = A.shape[0]
    lab = np.random.default_rng(seed).permutation(q)
    P = sp.csr_matrix((np.ones(q), (lab, np.arange(q))), shape=(q, q))
    B = (P @ A @ P.T).tocsr()
    B.sort_indices()
    return B


def test_rcm_and_min_degree_on_a_relabelled_path():
    """A path has no fill once numbered along itself (reverse Cuthill-McKee does that);
    minimum degree eliminates an end each time and fills nothing either; any order fills
    at most one entry per elimination (eliminating a vertex of a path leaves a path)."""
    q = 500
    A = sp.diags([np.ones(q - 1), np.ones(q), np.ones(q - 1)], [-1, 0, 1], format="csr")
    B = relabelled(A, 1)
    for order in (cg.CGGM_ORDER_RCM, cg.CGGM_ORDER_MINDEG):
        perm, parent, cc, nnz = cg.chol_symbolic(q, B.indptr, B.indices, order)
        assert np.array_equal(np.sort(perm), np.arange(q))
        assert nnz == 2 * q - 1
    _, _, _, nnz_nat = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_NATURAL)
    assert 2 * q - 1 <= nnz_nat <= 3 * q


def test_min_degree_has_no_fill_on_a_forest():
    """A forest always has a vertex of degree at most one, whose elimination creates no
    fill: nnz(L) = q + edges exactly."""
    rng = np.random.default_rng(10)
    q = 3000
    parent = np.array([rng.integers(0, v) if v > 0 and v % 50 else -1 for v in range(q)])
    child = np.flatnonzero(parent >= 0)
    A = sp.csr_matrix((np.ones(child.size), (child, parent[child])), shape=(q, q))
    B = relabelled((A + A.T).tocsr(), 4)
    perm, par, cc, nnz = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_MINDEG)
    assert np.array_equal(np.sort(perm), np.arange(q))
    assert nnz == q + child.size


def test_rcm_keeps_a_relabelled_band():
    """Bandwidth b: a band-preserving order fills only inside the band, at most
    (b + 1) entries per column."""
    q, b = 300, 4
    A = sp.diags([np.ones(q - abs(k)) for k in range(-b, b + 1)], list(range(-b, b + 1)),
                 format="csr")
    B = relabelled(A, 2)
    perm, parent, cc, nnz = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_RCM)
    assert np.array_equal(np.sort(perm), np.arange(q))
    assert cc.max() <= b + 1 and nnz <= q * (b + 1)


def test_tree_and_counts_are_consistent():
    """parent > k for every non-root; a column's count is at most its parent's + 1."""
    q = 400
    rp, ci = random_csr(q, 800, 8)
    perm, parent, cc, nnz = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_RCM)
    k = np.arange(q)
    nonroot = parent >= 0
    assert np.all(parent[nonroot] > k[nonroot])
    assert np.all(cc[nonroot] <= cc[parent[nonroot]] + 1)
    assert nnz == cc.sum() and np.all(cc >= 1)


def test_chain_with_links_at_the_largest_output_count():
    """q = 20000 outputs, a chain with random links (the block regime's network shape) on
    relabelled columns: minimum degree keeps the factor far sparser than the natural and
    the reverse Cuthill-McKee orders (which the long links defeat), within a second."""
    q = 20000
    rng = np.random.default_rng(9)
    for links in (200, 2000):
        i = np.r_[np.arange(q - 1), rng.integers(0, q, links)]
        j = np.r_[np.arange(1, q), rng.integers(0, q, links)]
        A = sp.csr_matrix((np.ones(i.size), (i, j)), shape=(q, q))
        B = relabelled((A + A.T).tocsr(), 3)
        t0 = time.perf_counter()
        _, _, _, nnz_md = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_MINDEG)
        assert time.perf_counter() - t0 < 5.0
        _, _, _, nnz_nat = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_NATURAL)
        _, _, _, nnz_rcm = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_RCM)
        assert 2 * q - 1 <= nnz_md < 0.5 * min(nnz_nat, nnz_rcm)


def test_min_degree_on_a_random_network():
    """A random network of average degree 4 (q = 2000): a valid order, counts consistent
    with the elimination tree, and less fill than the natural order."""
    q = 2000
    rp, ci = random_csr(q, 4000, 11)
    perm, parent, cc, nnz = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_MINDEG)
    assert np.array_equal(np.sort(perm), np.arange(q))
    nonroot = parent >= 0
    assert np.all(parent[nonroot] > np.arange(q)[nonroot])
    assert nnz == cc.sum()
    assert nnz < cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_NATURAL)[3]


def test_empty_and_errors():
    perm, parent, cc, nnz = cg.chol_symbolic(0, [0], [], cg.CGGM_ORDER_RCM)
    assert perm.size == 0 and nnz == 0
    rp, ci = np.array([0, 1, 2]), np.array([1, 0])
    with pytest.raises(cg.CGGMError):
        cg.chol_symbolic(2, rp, ci, 7)                                   # no such ordering
    with pytest.raises(cg.CGGMError):
        cg.chol_symbolic(2, rp, ci, cg.CGGM_ORDER_GIVEN, [0, 0])         # not a permutation
    with pytest.raises(cg.CGGMError):
        cg.chol_symbolic(2, rp, ci, cg.CGGM_ORDER_GIVEN)                 # no permutation given
    with pytest.raises(cg.CGGMError):
        cg.chol_symbolic(2, np.array([0, 1, 2]), np.array([1, 2]), cg.CGGM_ORDER_NATURAL)
    with pytest.raises(cg.CGGMError):
        cg.chol_symbolic(2, np.array([0, 2, 1]), np.array([1, 0]), cg.CGGM_ORDER_NATURAL)


@pytest.mark.parametrize("q,m,seed", [(1, 0, 12), (30, 25, 13), (80, 160, 14), (60, 900, 15)])
def test_supernodes_match_the_oracle(q, m, seed):
    rp, ci = random_csr(q, m, seed)
    rng = np.random.default_rng(seed)
    for perm in (np.arange(q), rng.permutation(q)):
        _, parent, cc, _ = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_GIVEN, perm)
        L = symbolic.cholesky_pattern(symbolic.pattern_from_csr(q, rp, ci), perm)
        assert np.array_equal(cg.chol_supernodes(parent, cc), symbolic.fundamental_supernodes(L))


def test_supernodes_of_a_dense_block_and_errors():
    q = 7
    A = sp.csr_matrix(np.ones((q, q)))
    _, parent, cc, _ = cg.chol_symbolic(q, A.indptr, A.indices, cg.CGGM_ORDER_NATURAL)
    assert cg.chol_supernodes(parent, cc).tolist() == [0, q]
    assert cg.chol_supernodes(np.zeros(0, np.int32), np.zeros(0, np.int64)).tolist() == [0]
    with pytest.raises(cg.CGGMError):
        cg.chol_supernodes([1, 0], [2, 1])          # a parent below its child
    with pytest.raises(cg.CGGMError):
        cg.chol_supernodes([1, -1], [3, 1])         # more entries than rows left


@pytest.mark.parametrize("q,m,seed", [(1, 1, 16), (25, 60, 17), (200, 900, 18)])
def test_permute_csr_is_the_definition(q, m, seed):
    """B[k][l] = A[perm[k]][perm[l]] entry for entry, columns ascending in every row."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, q, m)
    j = rng.integers(0, q, m)
    A = sp.csr_matrix((rng.standard_normal(m), (i, j)), shape=(q, q))
    A.sum_duplicates()
    perm = rng.permutation(q)
    rp, ci, v = cg.permute_csr(q, A.indptr, A.indices, A.data, perm)
    B = sp.csr_matrix((v, ci, rp), shape=(q, q))
    assert np.array_equal(B.toarray(), A.toarray()[np.ix_(perm, perm)])
    assert all(np.all(np.diff(ci[rp[k]:rp[k + 1]]) > 0) for k in range(q))
    # pattern only, and the inverse permutation restores A
    rp2, ci2, v2 = cg.permute_csr(q, A.indptr, A.indices, None, perm)
    assert v2 is None and np.array_equal(rp2, rp) and np.array_equal(ci2, ci)
    back = cg.permute_csr(q, rp, ci, v, np.argsort(perm))
    assert np.array_equal(back[0], A.indptr) and np.array_equal(back[1], A.indices)
    assert np.array_equal(back[2], A.data)


def test_permute_csr_errors():
    rp, ci, v = np.array([0, 1, 2]), np.array([1, 0]), np.array([1.0, 2.0])
    with pytest.raises(cg.CGGMError):
        cg.permute_csr(2, rp, ci, v, [1, 1])                  # not a permutation
    with pytest.raises(cg.CGGMError):
        cg.permute_csr(2, rp, np.array([1, 2]), v, [1, 0])    # column out of range


@pytest.mark.parametrize("q,m,seed", [(40, 50, 19), (90, 130, 20), (120, 1500, 21),
                                      (150, 6000, 22), (70, 0, 23)])
def test_min_degree_order_matches_the_oracle(q, m, seed):
    """The minimum-degree order is a definition with fixed tie-breaks, so the library's
    order equals the oracle's elimination game pivot for pivot, dense remainder included."""
    rp, ci = random_csr(q, m, seed)
    perm, _, _, _ = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_MINDEG)
    ref = symbolic.minimum_degree_order(symbolic.pattern_from_csr(q, rp, ci))
    assert np.array_equal(perm, ref)


@pytest.mark.parametrize("q,m,seed,order", [(1, 0, 24, 3), (30, 40, 25, 3), (80, 200, 26, 1),
                                            (60, 900, 27, 0), (120, 300, 28, 3)])
def test_supernode_rows_match_the_oracle(q, m, seed, order):
    """The rows of supernode s are the pattern of its first column in the oracle's factor."""
    rp, ci = random_csr(q, m, seed)
    perm, parent, cc, _ = cg.chol_symbolic(q, rp, ci, order)
    ss = cg.chol_supernodes(parent, cc)
    rows_ptr, rows = cg.chol_structure(q, rp, ci, perm, parent, cc, ss)
    L = symbolic.cholesky_pattern(symbolic.pattern_from_csr(q, rp, ci), perm)
    assert rows_ptr[-1] == sum(cc[ss[:-1]])
    for s in range(len(ss) - 1):
        assert np.array_equal(rows[rows_ptr[s]:rows_ptr[s + 1]], np.flatnonzero(L[:, ss[s]]))


def test_supernode_rows_reject_mismatched_inputs():
    q = 20
    rp, ci = random_csr(q, 30, 29)
    perm, parent, cc, _ = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_MINDEG)
    ss = cg.chol_supernodes(parent, cc)
    bad = cc.copy()
    bad[ss[0]] += 1 if bad[ss[0]] < q else -1
    with pytest.raises(cg.CGGMError):
        cg.chol_structure(q, rp, ci, perm, parent, bad, ss)
    with pytest.raises(cg.CGGMError):
        cg.chol_structure(q, rp, ci, perm, parent, cc, ss[::-1].copy())


def chain_with_links(q, links, seed=9):
    rng = np.random.default_rng(seed)
    i = np.r_[np.arange(q - 1), rng.integers(0, q, links)]
    j = np.r_[np.arange(1, q), rng.integers(0, q, links)]
    A = sp.csr_matrix((np.ones(i.size), (i, j)), shape=(q, q))
    return relabelled((A + A.T).tocsr(), 3)


def test_approximate_degrees_against_the_exact_order():
    """Approximate degrees bound the exact ones: the order is valid and its fill stays within
    a few percent of the exact minimum-degree order's on the same patterns (chains with
    links, a random network)."""
    cases = [chain_with_links(20000, 200), chain_with_links(20000, 2000)]
    rp, ci = random_csr(2000, 4000, 11)
    cases.append(sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(2000, 2000)))
    for B in cases:
        q = B.shape[0]
        perm, parent, cc, nnz_a = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_AMD)
        assert np.array_equal(np.sort(perm), np.arange(q))
        assert np.all(parent[parent >= 0] > np.arange(q)[parent >= 0])
        nnz_m = cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_MINDEG)[3]
        assert nnz_a <= 1.05 * nnz_m


def test_approximate_degrees_keep_a_forest_free_of_fill():
    rng = np.random.default_rng(10)
    q = 3000
    parent = np.array([rng.integers(0, v) if v > 0 and v % 50 else -1 for v in range(q)])
    child = np.flatnonzero(parent >= 0)
    A = sp.csr_matrix((np.ones(child.size), (child, parent[child])), shape=(q, q))
    B = relabelled((A + A.T).tocsr(), 4)
    assert cg.chol_symbolic(q, B.indptr, B.indices, cg.CGGM_ORDER_AMD)[3] == q + child.size


def test_approximate_degrees_at_the_block_regime_scale():
    """q = 100000 outputs, a chain with 10000 random links: the analysis takes seconds at
    most, where the exact order takes about 18 s."""
    B = chain_with_links(100000, 10000)
    t0 = time.perf_counter()
    perm, parent, cc, nnz = cg.chol_symbolic(100000, B.indptr, B.indices, cg.CGGM_ORDER_AMD)
    assert time.perf_counter() - t0 < 10.0
    assert np.array_equal(np.sort(perm), np.arange(100000))
    assert nnz == cc.sum()
