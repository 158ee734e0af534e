"""Equivariance pins of the oracle (CPU).  Eq. 1 is unchanged when the outputs are relabelled
(Lambda -> P Lambda P^T, Theta -> Theta P^T), when the inputs are relabelled (Theta's rows
permute), when outputs change sign (Lambda -> D Lambda D, Theta -> Theta D with D = diag(+-1);
the l1 norms do not change), and, with lambda_Theta = 0, when an input column is scaled by c
(its row of Theta scales by 1/c).  With n >= p + q + 10 the optimum is unique, so the oracle
must return the transformed optimum from the transformed data: an index, transpose or sign
slip anywhere in its passes, gradients or objective breaks one of these."""
import numpy as np

import oracle
import synth


def data(seed=41, p=5, q=4, n=40):
    pr = synth.make_problem(p, q, n, x_kind="gaussian", lam_kind="chain", theta_nnz=2,
                            lam=0.05, seed=seed)
    return pr.X, pr.Y


def solve(X, Y, lam_L=0.05, lam_T=0.05):
    return oracle.solve(X, Y, lam_L, lam_T, tol=1e-11, max_iter=4000)


def close(a, b, tol=2e-6):
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


def test_output_relabelling():
    X, Y = data()
    r = solve(X, Y)
    pi = np.array([2, 0, 3, 1])
    s = solve(X, Y[:, pi])
    assert abs(s.f - r.f) <= 1e-10 * abs(r.f)
    assert close(s.Lambda, r.Lambda[np.ix_(pi, pi)])
    assert close(s.Theta, r.Theta[:, pi])


def test_input_relabelling():
    X, Y = data(seed=42)
    r = solve(X, Y)
    pi = np.array([4, 2, 0, 1, 3])
    s = solve(X[:, pi], Y)
    assert abs(s.f - r.f) <= 1e-10 * abs(r.f)
    assert close(s.Lambda, r.Lambda)
    assert close(s.Theta, r.Theta[pi, :])


def test_output_sign_flips():
    X, Y = data(seed=43)
    r = solve(X, Y)
    d = np.array([1.0, -1.0, -1.0, 1.0])
    s = solve(X, Y * d)
    assert abs(s.f - r.f) <= 1e-10 * abs(r.f)
    assert close(s.Lambda, d[:, None] * r.Lambda * d[None, :])
    assert close(s.Theta, r.Theta * d[None, :])


def test_input_scaling_without_theta_penalty():
    """lambda_Theta = 0: scaling input k by c leaves Lambda and f unchanged and divides row
    k of Theta by c (with an l1 penalty on Theta this would not hold)."""
    X, Y = data(seed=44)
    r = solve(X, Y, lam_T=0.0)
    c = np.array([1.0, 3.0, 1.0, 0.25, 1.0])
    s = solve(X * c, Y, lam_T=0.0)
    assert abs(s.f - r.f) <= 1e-9 * abs(r.f)
    assert close(s.Lambda, r.Lambda)
    assert close(s.Theta, r.Theta / c[:, None])


def test_warm_start_at_the_optimum_stops_at_once():
    """Started from its own optimum, the method's stopping rule holds at the first check
    (the minimum-norm subgradient is already below tol times the l1 norms), so the solve
    returns that point with the same objective."""
    X, Y = data(seed=45)
    r = solve(X, Y)
    w = oracle.solve(X, Y, 0.05, 0.05, tol=1e-6, max_iter=50, Lambda0=r.Lambda,
                     Theta0=r.Theta)
    assert w.converged and w.iterations == 1
    assert np.array_equal(w.Lambda, r.Lambda) and np.array_equal(w.Theta, r.Theta)
    assert abs(w.f - r.f) <= 1e-14 * abs(r.f)
