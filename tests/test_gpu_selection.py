"""Model selection over the solver (Section 5: penalties chosen so that the estimated edge
counts match the true ones; cross-validation over a lambda path), every solve through the
C ABI."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
cg = pytest.importorskip("paper_1509_04681_gb300")
from paper_1509_04681_gb300 import selection  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    from paper_1509_04681_gb300 import build
    build.build()
    c = cg.Context(0)
    yield c
    c.close()


def test_penalties_for_the_true_edge_counts(ctx):
    pr = synth.make_problem(60, 40, 200, x_kind="gaussian", lam_kind="chain", theta_nnz=2,
                            lam=0.1, seed=41)
    e_L = int(np.count_nonzero(np.triu(pr.Lambda_true.toarray(), 1)))   # 39 chain edges
    e_T = int(pr.Theta_true.nnz)                                        # 80
    m = selection.lambdas_for_edges(ctx, pr.X, pr.Y, e_L, e_T, rel_tol=0.1,
                                    opts=cg.make_opts(precision=cg.CGGM_FP64))
    assert abs(m.edges_L - e_L) <= 0.1 * e_L and abs(m.edges_T - e_T) <= 0.1 * e_T, m
    assert (m.edges_L, m.edges_T) == selection.edge_counts(m.result)
    # with n = 200 samples the chain and Theta's support are recovered well at that size
    f_L = selection.support_f1(m.result.Lambda, pr.Lambda_true, upper=True).f1
    f_T = selection.support_f1(m.result.Theta, pr.Theta_true).f1
    assert f_L > 0.8 and f_T > 0.8, (f_L, f_T)


def test_cross_validation_over_a_path(ctx):
    pr = synth.make_problem(40, 20, 150, x_kind="gaussian", lam_kind="chain", theta_nnz=2,
                            lam=0.1, seed=42)
    lams = [0.5, 0.25, 0.12, 0.06, 0.03]
    cv = selection.cross_validate(ctx, pr.X, pr.Y, lams, folds=3,
                                  opts=cg.make_opts(precision=cg.CGGM_FP64))
    assert cv.loss.shape == (3, 5) and np.all(np.isfinite(cv.loss))
    # the heaviest penalty fits worst on held-out rows; the chosen lambda is one of the path's
    assert cv.mean[0] > cv.mean.min() and cv.best_lambda in lams
