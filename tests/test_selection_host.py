"""Host logic of the model-selection helpers (no GPU): edge counting and the F1 of a
recovered support, checked by hand."""
import types

import numpy as np
import pytest

from paper_1509_04681_gb300 import selection


def test_support_f1_by_hand():
    true = np.array([[2.0, 0.5, 0.0], [0.5, 2.0, 0.3], [0.0, 0.3, 2.0]])
    est = np.array([[1.9, 0.4, 0.1], [0.4, 2.1, 0.0], [0.1, 0.0, 2.0]])
    # Lambda edges (i < j): true {(0,1), (1,2)}, found {(0,1), (0,2)}: tp 1
    s = selection.support_f1(est, true, upper=True)
    assert (s.true_edges, s.found_edges) == (2, 2)
    assert s.precision == 0.5 and s.recall == 0.5 and s.f1 == 0.5
    # with a threshold that drops the 0.1 entry: found {(0,1)}, precision 1, recall 1/2
    s = selection.support_f1(est, true, threshold=0.2, upper=True)
    assert s.precision == 1.0 and s.recall == 0.5 and abs(s.f1 - 2 / 3) < 1e-15
    # all entries (Theta-like): 7 true nonzeros, 7 found, 5 in common
    s = selection.support_f1(est, true)
    assert (s.true_edges, s.found_edges) == (7, 7) and abs(s.f1 - 5 / 7) < 1e-15
    # nothing to find and nothing found
    z = selection.support_f1(np.zeros((2, 2)), np.zeros((2, 2)))
    assert z.precision == 1.0 and z.recall == 1.0 and z.f1 == 1.0
    with pytest.raises(ValueError):
        selection.support_f1(np.zeros((2, 2)), np.zeros((3, 3)))


def test_edge_counts_from_coordinate_lists():
    res = types.SimpleNamespace(
        Lambda_coo=(np.array([0, 0, 1, 1, 2], np.int32), np.array([0, 1, 1, 2, 2], np.int32),
                    np.array([2.0, 0.4, 2.0, -0.3, 2.0])),
        Theta_coo=(np.array([0, 3], np.int32), np.array([1, 0], np.int32), np.array([0.7, -1.0])))
    assert selection.edge_counts(res) == (2, 2)


class OracleContext:
    """Stands in for Context.cggm_solve on tiny problems: the oracle's Algorithm 1, warm
    starts given as coordinate lists as the binding passes them."""

    def __init__(self):
        self.calls = 0

    def cggm_solve(self, X, Y, lam_L, lam_T, tol=0.01, opts=None, warm_Lambda=None,
                   warm_Theta=None):
        import oracle
        self.calls += 1
        q, p = Y.shape[1], X.shape[1]
        L0 = T0 = None
        if warm_Lambda is not None:
            r, c, v = warm_Lambda
            L0 = np.zeros((q, q))
            L0[r, c] = v
            L0[c, r] = v
        if warm_Theta is not None:
            r, c, v = warm_Theta
            T0 = np.zeros((p, q))
            T0[r, c] = v
        res = oracle.solve(X, Y, lam_L, lam_T, tol=1e-6, max_iter=200, Lambda0=L0, Theta0=T0)
        iu = np.nonzero(np.triu(res.Lambda))
        it = np.nonzero(res.Theta)
        return types.SimpleNamespace(
            Lambda=res.Lambda, Theta=res.Theta,
            Lambda_coo=(iu[0].astype(np.int32), iu[1].astype(np.int32), res.Lambda[iu]),
            Theta_coo=(it[0].astype(np.int32), it[1].astype(np.int32), res.Theta[it]))


def test_recovery_versus_n_orchestration():
    """The study's host logic on a 5-output chain with 4 inputs, solved by the oracle: one
    point per n with the penalties' search count, supports scored against the true model,
    and near-perfect recovery once n is large."""
    import synth
    q, p = 5, 4
    Lt = synth.chain_precision(q).toarray()
    Tt = np.zeros((p, q))
    Tt[0, 1] = Tt[1, 3] = Tt[3, 0] = 1.0
    Tt[2, 4] = -1.0

    def sample(n, rng):
        X = rng.standard_normal((n, p))
        return X, synth.sample_Y(X, Tt, Lt, rng)

    ctx = OracleContext()
    pts = selection.recovery_versus_n(ctx, sample, Lt, Tt, [40, 2000], seed=3, rounds=25)
    assert [pt.n for pt in pts] == [40, 2000]
    assert sum(pt.solves for pt in pts) == ctx.calls
    for pt in pts:
        assert pt.lambda_support.true_edges == 4 and pt.theta_support.true_edges == 4
        assert 0.0 <= pt.lambda_support.f1 <= 1.0 and pt.lam_L > 0 and pt.lam_T > 0
    big = pts[-1]
    assert big.lambda_support.f1 >= 0.85 and big.theta_support.f1 >= 0.85
