"""The numeric sparse Cholesky (cggm_spchol_*) through the C ABI, against the oracle.

Section 4 keeps Lambda sparse in the block regime, and the Armijo rule needs log det of a
sparse positive definite matrix and its positive definiteness, which a sparse factor
gives; columns of Sigma = Lambda^-1 come from two triangular solves with it.  The factor
P A P^T = L L^T is unique, so the GPU's supernodal blocks are compared entry by entry with
the oracle's definition (LAPACK's dense factor of the permuted matrix), log det with the
oracle's, and the solves with the oracle's spd_solve.  Cases: chains with random links and
random networks under every pivot order, a forest, a diagonal matrix, a dense matrix (one
supernode), a star whose centre updates a 1100-column supernode (more rows than one map
chunk), q = 1, matrices that are not positive definite or not finite, and tridiagonal
Toeplitz matrices at q = 200000 against their closed-form determinants.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1509_04681_gb300")

ORDERS = [cg.CGGM_ORDER_NATURAL, cg.CGGM_ORDER_RCM, cg.CGGM_ORDER_MINDEG, cg.CGGM_ORDER_AMD]


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_04681_gb300 import build
    build.build()
    c = cg.Context(0)
    yield c
    c.close()


def lower_csr(A):
    """CSR of the lower triangle with the diagonal (the values the factor reads)."""
    m = sp.tril(sp.csr_matrix(A)).tocsr()
    m.sort_indices()
    return m


def check_factor(ctx, A, ordering, perm=None, full=False):
    """Factor A (dense symmetric) on the GPU; compare L, log det and a solve with the oracle."""
    m = sp.csr_matrix(A) if full else lower_csr(A)
    with ctx.cggm_spchol(m.indptr, m.indices, ordering, perm) as f:
        ld = f.factor(m.data)
        e = f.export()
        Lg = f.dense_factor()
        Lo, ldo = oracle.symbolic.numeric_factor(A, e["perm"])
        scale = np.max(np.abs(Lo))
        assert np.max(np.abs(Lg - Lo)) <= 1e-12 * scale
        assert abs(ld - ldo) <= 1e-12 * max(1.0, abs(ldo))
        q = A.shape[0]
        k = min(q, 7)
        c0 = q // 3 if q > k else 0
        X = f.solve(c0=c0, k=k)  # columns c0 .. c0 + k - 1 of A^-1
        E = np.zeros((q, k))
        E[c0 + np.arange(k), np.arange(k)] = 1.0
        Xo = oracle.spd_solve(A, E)
        assert np.max(np.abs(X - Xo)) <= 1e-10 * np.max(np.abs(Xo))
        B = np.random.default_rng(1).standard_normal((q, 3))
        np.testing.assert_allclose(f.solve(B), oracle.spd_solve(A, B), rtol=0,
                                   atol=1e-10 * np.max(np.abs(oracle.spd_solve(A, B))))
        return e


@pytest.mark.parametrize("ordering", ORDERS)
def test_chain_with_links(ctx, ordering):
    rng = np.random.default_rng(3)
    q = 600
    A = synth.random_sparse_precision(q, 1.0, rng, base=synth.chain_precision(q)).toarray()
    check_factor(ctx, A, ordering)


@pytest.mark.parametrize("ordering", [cg.CGGM_ORDER_AMD, cg.CGGM_ORDER_MINDEG])
def test_random_network_and_clustered(ctx, ordering):
    rng = np.random.default_rng(4)
    A = synth.random_sparse_precision(500, 4.0, rng).toarray()
    e = check_factor(ctx, A, ordering)
    assert e["nsuper"] < 500  # fill joins columns into supernodes wider than one
    C = synth.clustered_precision(750, np.random.default_rng(5)).toarray()
    check_factor(ctx, C, ordering)


def test_given_order_and_both_triangles(ctx):
    rng = np.random.default_rng(6)
    q = 300
    A = synth.random_sparse_precision(q, 3.0, rng).toarray()
    perm = rng.permutation(q).astype(np.int32)
    e = check_factor(ctx, A, cg.CGGM_ORDER_GIVEN, perm=perm, full=True)
    np.testing.assert_array_equal(e["perm"], perm)


def test_degenerate_shapes(ctx):
    check_factor(ctx, np.array([[2.5]]), cg.CGGM_ORDER_AMD)                  # q = 1
    check_factor(ctx, np.diag(np.arange(1.0, 41.0)), cg.CGGM_ORDER_NATURAL)  # no edges
    rng = np.random.default_rng(7)
    # a forest: a chain of 100 and a star of 50, disconnected
    F = synth.chain_precision(150).toarray()
    F[99, 100] = F[100, 99] = 0.0
    F[100:, 100:] = 0.0
    F[100, 101:] = F[101:, 100] = 0.1
    F[np.arange(100, 150), np.arange(100, 150)] = 6.0
    e = check_factor(ctx, F, cg.CGGM_ORDER_MINDEG)
    assert e["nnz_L"] == np.count_nonzero(np.tril(F))  # minimum degree: no fill on a forest
    D = rng.standard_normal((60, 70))
    check_factor(ctx, D @ D.T / 70 + np.eye(60), cg.CGGM_ORDER_NATURAL)     # dense


def test_update_wider_than_one_map_chunk(ctx):
    """Pivot 0 is the centre of a star over pivots 2 .. 1101 and pivot 1 touches pivot 2
    only: pivot 2 then has two children, so pivots 2 .. 1101 (a clique after eliminating
    the centre) form their own supernode, updated by the centre's 1100 rows."""
    q = 1102
    A = np.eye(q) * 3.0
    A[0, 0] = 1200.0
    A[0, 2:] = A[2:, 0] = 1.0
    A[1, 2] = A[2, 1] = 0.5
    e = check_factor(ctx, A, cg.CGGM_ORDER_NATURAL)
    ss = e["super_start"]
    assert list(ss[:3]) == [0, 1, 2] and ss[3] == q


def test_deterministic_bits(ctx):
    rng = np.random.default_rng(8)
    A = synth.random_sparse_precision(2000, 3.0, rng, base=synth.chain_precision(2000))
    m = lower_csr(A.toarray())
    with ctx.cggm_spchol(m.indptr, m.indices) as f:
        l1 = f.factor(m.data)
        b1 = f.export()["blocks"].copy()
        l2 = f.factor(m.data)
        b2 = f.export()["blocks"]
    assert l1 == l2
    np.testing.assert_array_equal(b1, b2)


def test_not_positive_definite_and_not_finite(ctx):
    q = 50
    A = synth.chain_precision(q, diag=1.0, off=0.6).toarray()  # indefinite (0.6 > 1/2)
    m = lower_csr(A)
    with ctx.cggm_spchol(m.indptr, m.indices) as f:
        with pytest.raises(cg.CGGMError) as ex:
            f.factor(m.data)
        assert ex.value.status == cg.CGGM_ENOTPD
        with pytest.raises(cg.CGGMError) as ex:
            f.solve(c0=0, k=1)  # no successful factorisation
        assert ex.value.status == cg.CGGM_EINVAL
        bad = m.data.copy()
        bad[3] = np.nan
        with pytest.raises(cg.CGGMError) as ex:
            f.factor(bad)
        assert ex.value.status == cg.CGGM_ENONFINITE
        good = lower_csr(synth.chain_precision(q).toarray())
        assert np.isfinite(f.factor(good.data))  # same pattern, usable again
    with pytest.raises(cg.CGGMError) as ex:
        ctx.cggm_spchol(np.array([0, 1, 3]), np.array([0, 0, 5]))  # column outside [0, q)
    assert ex.value.status == cg.CGGM_EINVAL


def relabelled_tridiagonal(q, diag, lab):
    """Lower triangle (CSR) of the tridiagonal Toeplitz matrix with `diag` on the diagonal and
    -1 beside it, its path relabelled by the permutation lab."""
    i = np.arange(q - 1)
    r = np.concatenate([lab, lab[i + 1]])
    c = np.concatenate([lab, lab[i]])
    v = np.concatenate([np.full(q, float(diag)), np.full(q - 1, -1.0)])
    m = sp.csr_matrix((v, (np.maximum(r, c), np.minimum(r, c))), shape=(q, q))
    m.sort_indices()
    return m


def test_tridiagonal_closed_forms_at_scale(ctx):
    """q = 200000 (the block regime's largest output count), labels permuted at random so
    that the pivot order matters.  The eigenvalues of the tridiagonal Toeplitz matrix
    T_a = tridiag(-1, a, -1) are a - 2 cos(k pi / (q + 1)), k = 1 .. q, so log det T_a is
    their log sum; for a = 2 (the second-difference matrix) that is log(q + 1), and
    (T_2^-1)_ij = min(i, j) (q + 1 - max(i, j)) / (q + 1) (1-based).
    Tolerances: T_3 has condition number below 5, so log det and the solve are within a few
    hundred roundings.  T_2 has condition number ~0.4 q^2 = 1.6e10: the factorisation's
    backward error E (entries ~3 eps |L| |L^T|) moves log det by tr(T_2^-1 E), a sum of q
    terms of random sign with (T_2^-1)_ii up to q / 4, ~1e-8 here; the solve is accurate to
    the condition number times eps relative to its largest entry (~2e-6)."""
    q = 200000
    rng = np.random.default_rng(9)
    lab = rng.permutation(q)
    k = np.arange(1, q + 1)
    for diag in (3.0, 2.0):
        m = relabelled_tridiagonal(q, diag, lab)
        # (for a = 2 the closed form: the product formula loses digits to 2 - 2 cos(small))
        want_ld = (np.log(q + 1) if diag == 2.0
                   else float(np.sum(np.log(diag - 2.0 * np.cos(k * np.pi / (q + 1))))))
        for ordering in (cg.CGGM_ORDER_AMD, cg.CGGM_ORDER_RCM):
            with ctx.cggm_spchol(m.indptr, m.indices, ordering) as f:
                ld = f.factor(m.data)
                assert abs(ld - want_ld) <= (1e-9 if diag == 3.0 else 1e-7)
                assert f.export(blocks=False)["nnz_L"] == 2 * q - 1  # a path: no fill
                j = 777
                x = f.solve(c0=int(lab[j]), k=1)[:, 0]
                # residual in original labels: T x = e_j
                full = m + sp.tril(m, -1).T
                res = full @ x
                res[lab[j]] -= 1.0
                assert np.max(np.abs(res)) <= 1e-10 * np.max(np.abs(x)) * (diag + 2)
                if diag == 2.0:
                    t = np.arange(q)
                    want = (np.minimum(t, j) + 1.0) * (q - np.maximum(t, j)) / (q + 1)
                    np.testing.assert_allclose(x[lab], want, rtol=0, atol=1e-5 * want.max())
