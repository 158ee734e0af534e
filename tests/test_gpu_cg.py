"""Sparse SPD solves by conjugate gradient through the C ABI (Section 4: columns of
Sigma = Lambda^-1 and P = R Sigma from the sparse Lambda), against the oracle's
definition X = Lambda^-1 B (needs a GPU)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import synth

pytestmark = pytest.mark.gpu

cg = pytest.importorskip("paper_1509_04681_gb300")


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_04681_gb300 import build
    build.build()
    c = cg.Context(0)
    yield c
    c.close()


def rel(a, b):
    return np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)))


def csr(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


@pytest.mark.parametrize("kind,q", [("chain", 300), ("random4", 500), ("chain", 5000)])
def test_sigma_columns(ctx, kind, q):
    rng = np.random.default_rng(1)
    Lam = synth.chain_precision(q) if kind == "chain" else synth.random_sparse_precision(q, 4, rng)
    c0, k = 17, 40
    X, iters, res = ctx.cggm_spd_solve(*csr(Lam), c0=c0, k=k, tol=1e-12, max_iter=2000)
    E = np.zeros((q, k))
    E[c0 + np.arange(k), np.arange(k)] = 1.0
    ref = oracle.spd_solve(Lam.toarray(), E)
    assert res <= 1e-12 and 0 < iters < 2000
    assert rel(X, ref) < 1e-9


def test_general_right_hand_sides_and_P(ctx):
    """Lambda P^T = R^T gives P = R Sigma (R = X Theta of a generated problem)."""
    pr = synth.make_problem(60, 200, 50, lam_kind="random4", seed=2, theta_nnz=3)
    Lam = pr.Lambda_true
    R = pr.X @ pr.Theta_true.toarray()
    Pt, iters, res = ctx.cggm_spd_solve(*csr(Lam), B=R.T.copy(), tol=1e-12, max_iter=2000)
    ref = oracle.spd_solve(Lam.toarray(), R.T)
    assert rel(Pt, ref) < 1e-9
    Sigma = oracle.spd_solve(Lam.toarray(), np.eye(200))
    assert rel(Pt.T, R @ Sigma) < 1e-9


def test_zero_rhs_and_iteration_limit(ctx):
    Lam = synth.chain_precision(100)
    X, iters, res = ctx.cggm_spd_solve(*csr(Lam), B=np.zeros((100, 3)), tol=1e-10)
    assert iters == 0 and res == 0.0 and np.all(X == 0.0)
    X, iters, res = ctx.cggm_spd_solve(*csr(Lam), c0=0, k=2, tol=1e-14, max_iter=2,
                                       allow_maxiter=True)
    assert iters == 2 and res > 1e-14


def test_not_positive_definite_and_malformed(ctx):
    ind = csr(np.array([[1.0, 2.0], [2.0, 1.0]]))  # positive diagonal, indefinite
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_spd_solve(*ind, c0=0, k=1, tol=1e-12)
    assert e.value.status == cg.CGGM_ENOTPD
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_spd_solve(*csr(np.diag([1.0, -1.0])), c0=0, k=2, tol=1e-12)
    assert e.value.status == cg.CGGM_ENOTPD
    rp, ci, va = csr(synth.chain_precision(10))
    bad = ci.copy()
    bad[3] = 10  # column outside [0, q)
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_spd_solve(rp, bad, va, c0=0, k=1, tol=1e-12)
    assert e.value.status == cg.CGGM_EINVAL


@pytest.mark.parametrize("kind", ["chain", "random4"])
def test_lambda_gradient_column_block(ctx, kind):
    """G_Lambda[:, C] from the sparse Lambda by conjugate gradient (Sigma never formed) against
    the oracle's full gradient of Eq. 3."""
    pr = synth.make_problem(80, 300, 60, lam_kind=kind, seed=4, theta_nnz=3)
    Lam = pr.Lambda_true
    Th = 0.5 * pr.Theta_true.toarray()
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    G_L, _, _, _ = oracle.gradients(Lam.toarray(), Th, Sxx, Sxy, Syy)
    for c0, k in ((0, 64), (250, 50), (123, 1)):
        G, iters = ctx.cggm_grad_lambda_block(pr.X, pr.Y, *csr(Lam), Th, c0, k, tol=1e-12,
                                              max_iter=3000)
        assert 0 < iters < 3000
        assert rel(G, G_L[:, c0:c0 + k]) < 1e-9
    with pytest.raises(cg.CGGMError):
        ctx.cggm_grad_lambda_block(pr.X, pr.Y, *csr(Lam), Th, 290, 20)
