"""Prediction with a fitted model (cggm_predict, Section 2.1: E[y | x] = -Lambda^-1 Theta^T x,
B = -Theta Sigma) through the C ABI, against the oracle's plain definition."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("x_kind", ["gaussian", "genotype"])
def test_predict_matches_oracle_on_a_solved_model(ctx, x_kind):
    pr = synth.make_problem(150, 70, 90, x_kind=x_kind, lam_kind="random4", theta_nnz=4,
                            lam=0.1, seed=31)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-4,
                       opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=500))
    # the returned coordinate lists in, predictions for new inputs out
    Xnew = synth.make_problem(150, 70, 40, x_kind=x_kind, lam_kind="random4", theta_nnz=4,
                              lam=0.1, seed=32).X
    Yh, B = ctx.cggm_predict(Xnew, r.Lambda_coo, r.Theta_coo, q=70)
    Yh_ref, B_ref = oracle.predict(Xnew, r.Lambda, r.Theta)
    assert rel(B, B_ref) < 1e-10 and rel(Yh, Yh_ref) < 1e-10
    # dense matrices in (marshalled to coordinate lists), only B wanted
    _, B2 = ctx.cggm_predict(Xnew, r.Lambda, r.Theta)
    np.testing.assert_array_equal(B2, B)


def test_predict_genotype_counts_are_standardised(ctx):
    """int8 counts are standardised per column on the device, as cggm_solve does."""
    pr = synth.make_problem(60, 20, 50, x_kind="genotype", lam_kind="chain", theta_nnz=3,
                            lam=0.1, seed=33)
    Lam = np.linalg.inv(np.cov(pr.Y.T) + 0.5 * np.eye(20))
    Th = np.zeros((60, 20))
    Th[np.arange(20) * 3, np.arange(20)] = 0.7
    Yh8, _ = ctx.cggm_predict(pr.X_raw, Lam, Th, want_B=False)
    Yh_ref, _ = oracle.predict(pr.X, Lam, Th)
    assert rel(Yh8, Yh_ref) < 1e-10


def test_predict_errors(ctx):
    X = np.ones((5, 3))
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_predict(X, -np.eye(2), np.zeros((3, 2)))
    assert e.value.status == cg.CGGM_ENOTPD
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_predict(X, (np.array([1]), np.array([0]), np.array([1.0])),
                         (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0)), q=2)
    assert e.value.status == cg.CGGM_EINVAL  # an entry below the diagonal of Lambda
