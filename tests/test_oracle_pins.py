"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: a closed form, a
reduction to a textbook problem solved by a different algorithm, finite differences
of Eq. 1, or brute-force minimisation.  Together they are chosen so that a dropped
term, a wrong sign or index, or a missing factor anywhere in the oracle fails one.
"""
import numpy as np
import pytest
import scipy.optimize as so

import oracle
import synth
from tests import bruteforce as bf

pytestmark = []


def small_problem(p, q, n, seed, lam_kind="chain", x_kind="gaussian", theta_nnz=2):
    pr = synth.make_problem(p, q, n, x_kind=x_kind, lam_kind=lam_kind, theta_nnz=theta_nnz,
                            lam=0.1, seed=seed)
    return pr.X, pr.Y


def tight_solve(X, Y, lam_L, lam_T, **kw):
    """Run the oracle far past the paper's stopping ratio.  Close to the optimum the
    Armijo test meets the rounding of f (changes near 1e-16 |f|), where progress stops;
    parameters are then accurate to about 1e-8 relative, which the pins allow for."""
    kw.setdefault("max_iter", 3000)
    return oracle.solve(X, Y, lam_L, lam_T, tol=1e-11, **kw)


# --------------------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------------------

def test_lambda_zero_closed_form():
    """lambda = 0 with n >= p + q: stationarity of Eq. 1 gives
    Lambda = (S_yy - S_xy^T S_xx^-1 S_xy)^-1, Theta = -S_xx^-1 S_xy Lambda."""
    X, Y = small_problem(6, 4, 60, seed=3)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    Lam_cf = np.linalg.inv(Syy - Sxy.T @ np.linalg.solve(Sxx, Sxy))
    Th_cf = -np.linalg.solve(Sxx, Sxy) @ Lam_cf
    r = oracle.solve(X, Y, 0.0, 0.0, tol=1e-13, max_iter=20000)
    assert r.converged
    assert np.max(np.abs(r.Lambda - Lam_cf)) < 1e-8 * np.max(np.abs(Lam_cf))
    assert np.max(np.abs(r.Theta - Th_cf)) < 1e-8 * np.max(np.abs(Th_cf))


def test_scalar_closed_form():
    """p = q = 1: with u = max(|s_xy| - lam_T/2, 0), Lambda = 1/(s_yy - u^2/s_xx + lam_L)
    and Theta = -Lambda sign(s_xy) u / s_xx (minimising Eq. 1 in two scalars)."""
    rng = np.random.default_rng(0)
    for trial in range(5):
        x = rng.standard_normal((40, 1))
        y = -0.8 * x + 0.5 * rng.standard_normal((40, 1))
        lam_L, lam_T = 0.05 * (trial + 1), 0.1 * trial
        sxx, sxy, syy = (float((a.T @ b)[0, 0]) / 40 for a, b in ((x, x), (x, y), (y, y)))
        u = max(abs(sxy) - lam_T / 2, 0.0)
        Lam = 1.0 / (syy - u * u / sxx + lam_L)
        Th = -Lam * np.sign(sxy) * u / sxx
        # near the optimum the Armijo test runs into the rounding of f (changes of
        # 1e-17), which limits the attainable accuracy of the parameters to ~1e-8
        r = oracle.solve(x, y, lam_L, lam_T, tol=1e-12, max_iter=400)
        assert abs(r.Lambda[0, 0] - Lam) < 1e-7 * Lam
        assert abs(r.Theta[0, 0] - Th) < 1e-7 * max(1.0, abs(Th))


def test_q1_reduces_to_lasso():
    """q = 1: substituting Theta = -Lambda w turns Eq. 1 into
    -log L + L [(1/n)||y - Xw||^2 + lam_T ||w||_1 + lam_L], so w is the Lasso solution
    and Lambda = 1 / (Lasso optimum + lam_L)."""
    X, Y = small_problem(12, 1, 50, seed=7, theta_nnz=3)
    lam_L, lam_T = 0.07, 0.15
    w = bf.lasso_cd(X, Y[:, 0], lam_T)
    val = np.mean((Y[:, 0] - X @ w) ** 2) + lam_T * np.abs(w).sum()
    Lam = 1.0 / (val + lam_L)
    r = tight_solve(X, Y, lam_L, lam_T)
    assert abs(r.Lambda[0, 0] - Lam) < 1e-7 * Lam
    np.testing.assert_allclose(r.Theta[:, 0], -Lam * w, atol=1e-6 * np.abs(w).max())
    # same support
    assert set(np.flatnonzero(np.abs(r.Theta[:, 0]) > 1e-9)) == set(np.flatnonzero(np.abs(w) > 1e-9))


def test_q1_matches_sklearn_lasso():
    sk = pytest.importorskip("sklearn.linear_model")
    X, Y = small_problem(15, 1, 60, seed=11, theta_nnz=4)
    lam_L, lam_T = 0.02, 0.2
    m = sk.Lasso(alpha=lam_T / 2, fit_intercept=False, tol=1e-14, max_iter=200000).fit(X, Y[:, 0])
    w = m.coef_
    Lam = 1.0 / (np.mean((Y[:, 0] - X @ w) ** 2) + lam_T * np.abs(w).sum() + lam_L)
    r = tight_solve(X, Y, lam_L, lam_T)
    assert abs(r.Lambda[0, 0] - Lam) < 1e-7 * Lam
    np.testing.assert_allclose(r.Theta[:, 0], -Lam * w, atol=1e-6 * np.abs(w).max())


def test_theta_zero_regime_is_graphical_lasso():
    """lam_T >= 2 max|S_xy| makes Theta = 0 optimal (its gradient 2 S_xy is inside the
    l1 ball at Theta = 0 for any Lambda); Lambda then solves the graphical lasso on S_yy
    with the diagonal penalised.  Checked against a brute-force proximal solver."""
    X, Y = small_problem(5, 5, 30, seed=5)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    lam_T = 2.0 * np.abs(Sxy).max() * 1.01
    lam_L = 0.1
    r = tight_solve(X, Y, lam_L, lam_T)
    assert np.all(r.Theta == 0)
    Xz = np.zeros_like(X[:, :1])
    L_bf, T_bf, f_bf = bf.fista_cggm(Xz, Y, lam_L, 1.0, iters=30000)
    np.testing.assert_allclose(r.Lambda, L_bf, atol=1e-6)


# --------------------------------------------------------------------------------------
# derivatives of Eq. 1
# --------------------------------------------------------------------------------------

def test_gradient_finite_differences():
    """Eq. 3 against central differences of Eq. 1 along random symmetric (Lambda) and
    arbitrary (Theta) directions."""
    X, Y = small_problem(7, 5, 40, seed=1)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    rng = np.random.default_rng(1)
    Lam = np.eye(5) + 0.1 * (lambda A: A + A.T)(rng.standard_normal((5, 5)))
    Th = rng.standard_normal((7, 5)) * 0.3
    G_L, G_T, _, _ = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    g = lambda L, T: bf.cggm_f(L, T, X, Y, 0.0, 0.0)  # noqa: E731
    h = 1e-5
    for _ in range(4):
        E = rng.standard_normal((5, 5)); E = E + E.T
        fd = (g(Lam + h * E, Th) - g(Lam - h * E, Th)) / (2 * h)
        assert abs(fd - np.sum(G_L * E)) < 1e-6 * max(1.0, abs(fd))
        F = rng.standard_normal((7, 5))
        fd = (g(Lam, Th + h * F) - g(Lam, Th - h * F)) / (2 * h)
        assert abs(fd - np.sum(G_T * F)) < 1e-6 * max(1.0, abs(fd))


def _model_value(Dm, G, Sigma, Psi):
    # second-order model, with its quadratic term pinned separately by test_hessian_*
    return np.sum(G * Dm) + 0.5 * np.trace(Sigma @ Dm @ Sigma @ Dm) + np.trace(Psi @ Dm @ Sigma @ Dm)


def test_hessian_quadratic_form_second_differences():
    """The quadratic term 1/2 tr(S D S D) + tr(P D S D) of the Lambda model equals half
    the second directional derivative of Eq. 1's smooth part (Eq. 4 as a quadratic form
    on symmetric D)."""
    X, Y = small_problem(6, 4, 50, seed=2)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    rng = np.random.default_rng(2)
    Lam = np.eye(4) + 0.15 * (lambda A: A + A.T)(rng.standard_normal((4, 4)))
    Th = rng.standard_normal((6, 4)) * 0.4
    G_L, _, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    g = lambda L: bf.cggm_f(L, Th, X, Y, 0.0, 0.0)  # noqa: E731
    h = 1e-4
    for _ in range(4):
        E = rng.standard_normal((4, 4)); E = E + E.T
        d2 = (g(Lam + h * E) - 2 * g(Lam) + g(Lam - h * E)) / h ** 2
        quad = _model_value(E, 0 * G_L, Sigma, Psi)
        assert abs(0.5 * d2 - quad) < 1e-5 * max(1.0, abs(quad))


# --------------------------------------------------------------------------------------
# coordinate steps by one-dimensional brute force
# --------------------------------------------------------------------------------------

def _brute_1d(fun, scale):
    best = None
    for lo, hi in [(-scale, scale), (-10 * scale, 10 * scale)]:
        r = so.minimize_scalar(fun, bounds=(lo, hi), method="bounded",
                               options={"xatol": 1e-13 * scale, "maxiter": 10000})
        if best is None or r.fun < best.fun:
            best = r
    # the optimum may sit at the kink where the l1 term vanishes; compare against it too
    return best.x, best.fun


@pytest.mark.parametrize("mutant", [False, True])
def test_lambda_coordinate_steps_brute_force(mutant):
    """Every step of the Lambda pass minimises the l1-regularised model exactly along
    its coordinate (E_ij + E_ji off the diagonal, E_ii on it).  With the curvature as
    printed in Appendix A.1 (mutant build), the steps are not minimisers."""
    X, Y = small_problem(6, 5, 40, seed=4)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    rng = np.random.default_rng(4)
    Lam = np.eye(5) + 0.2 * np.diag(np.ones(4), 1) + 0.2 * np.diag(np.ones(4), -1)
    Th = np.where(rng.uniform(size=(6, 5)) < 0.4, rng.standard_normal((6, 5)), 0.0)
    G_L, _, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    lam = 0.05
    coords = [(i, j) for i in range(5) for j in range(i, 5)]
    li = np.array([c[0] for c in coords], dtype=np.int32)
    lj = np.array([c[1] for c in coords], dtype=np.int32)
    worst = 0.0
    for k in range(len(coords)):
        D_before = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li[:k], lj[:k], lam, mutant=mutant)
        D_after = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li[:k + 1], lj[:k + 1], lam, mutant=mutant)
        i, j = coords[k]
        E = np.zeros((5, 5)); E[i, j] = 1.0; E[j, i] = 1.0
        phi = lambda t: _model_value(D_before + t * E, G_L, Sigma, Psi) + \
            lam * np.abs(Lam + D_before + t * E).sum()  # noqa: E731
        t_bf, f_bf = _brute_1d(phi, 2.0)
        t_or = D_after[i, j] - D_before[i, j]
        # compare objective values (robust at kinks) and the step itself
        worst = max(worst, phi(t_or) - f_bf)
        if not mutant:
            assert phi(t_or) <= f_bf + 1e-12
            assert abs(t_or - t_bf) < 1e-6
    if mutant:
        assert worst > 1e-8, "printed curvature was not caught"


@pytest.mark.parametrize("mutant", [False, True])
def test_theta_coordinate_steps_brute_force(mutant):
    """Every step of the Theta pass minimises Eq. 1 itself (Lambda fixed) exactly along
    E_ij.  The objective here is the independent autograd-free evaluation of Eq. 1."""
    X, Y = small_problem(6, 4, 40, seed=6)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    Lam = np.eye(4) + 0.3 * np.diag(np.ones(3), 1) + 0.3 * np.diag(np.ones(3), -1)
    Sigma = np.linalg.inv(Lam)
    rng = np.random.default_rng(6)
    Th0 = np.where(rng.uniform(size=(6, 4)) < 0.3, rng.standard_normal((6, 4)), 0.0)
    lam_T = 0.08
    coords = [(i, j) for i in range(6) for j in range(4)]
    ti = np.array([c[0] for c in coords], dtype=np.int32)
    tj = np.array([c[1] for c in coords], dtype=np.int32)
    worst = 0.0
    for k in range(len(coords)):
        Tb = oracle.theta_sweep(Sxx, Sxy, Sigma, Th0, ti[:k], tj[:k], lam_T, mutant=mutant)
        Ta = oracle.theta_sweep(Sxx, Sxy, Sigma, Th0, ti[:k + 1], tj[:k + 1], lam_T, mutant=mutant)
        i, j = coords[k]
        E = np.zeros((6, 4)); E[i, j] = 1.0
        phi = lambda t: bf.cggm_f(Lam, Tb + t * E, X, Y, 0.0, lam_T)  # noqa: E731
        t_bf, f_bf = _brute_1d(phi, 3.0)
        t_or = Ta[i, j] - Tb[i, j]
        worst = max(worst, phi(t_or) - f_bf)
        if not mutant:
            assert phi(t_or) <= f_bf + 1e-11
            assert abs(t_or - t_bf) < 1e-6
    if mutant:
        assert worst > 1e-8, "printed curvature was not caught"


# --------------------------------------------------------------------------------------
# whole-solver properties
# --------------------------------------------------------------------------------------

def test_tiny_problems_match_bruteforce_fista():
    """Convexity: the oracle and an accelerated proximal-gradient method on (Lambda,
    Theta) jointly reach the same optimum on tiny inputs."""
    for seed, (p, q, n) in enumerate([(4, 3, 20), (6, 5, 15), (3, 6, 25)]):
        X, Y = small_problem(p, q, n, seed=20 + seed)
        lam_L, lam_T = 0.12, 0.2
        r = tight_solve(X, Y, lam_L, lam_T)
        L_bf, T_bf, f_bf = bf.fista_cggm(X, Y, lam_L, lam_T, iters=60000)
        f_or = bf.cggm_f(r.Lambda, r.Theta, X, Y, lam_L, lam_T)
        assert abs(f_or - f_bf) <= 1e-9 * abs(f_bf)
        assert f_or <= f_bf + 1e-9 * abs(f_bf)
        assert np.max(np.abs(r.Lambda - L_bf)) < 1e-4
        assert np.max(np.abs(r.Theta - T_bf)) < 1e-4


def test_kkt_and_monotone_decrease():
    """At the returned point the subgradient conditions of Eq. 1 hold; along the way f
    never increases and Lambda stays positive definite."""
    X, Y = small_problem(20, 10, 30, seed=9, theta_nnz=3)
    lam_L, lam_T = 0.1, 0.15
    fs = []

    def cb(rec, Lam, Th):
        np.linalg.cholesky(Lam)
        fs.append(bf.cggm_f(Lam, Th, X, Y, lam_L, lam_T))

    r = tight_solve(X, Y, lam_L, lam_T, callback=cb)
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(fs, fs[1:]))
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    G_L, G_T, _, _ = oracle.gradients(r.Lambda, r.Theta, Sxx, Sxy, Syy)
    eps = 1e-7
    for G, P, lam in [(G_L, r.Lambda, lam_L), (G_T, r.Theta, lam_T)]:
        nz = P != 0
        assert np.all(np.abs(G[nz] + lam * np.sign(P[nz])) <= eps)
        assert np.all(np.abs(G[~nz]) <= lam + eps)


def test_objective_matches_independent_evaluation():
    X, Y = small_problem(9, 6, 25, seed=12)
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    rng = np.random.default_rng(12)
    Lam = np.eye(6) * 1.5 + 0.2 * np.diag(np.ones(5), 1) + 0.2 * np.diag(np.ones(5), -1)
    Th = rng.standard_normal((9, 6))
    for pen in (True, False):
        f_or = oracle.objective(Lam, Th, Sxx, Sxy, Syy, 0.3, 0.2, penalize_diag=pen)
        f_bf = bf.cggm_f(Lam, Th, X, Y, 0.3, 0.2, penalize_diag=pen)
        assert abs(f_or - f_bf) < 1e-12 * abs(f_bf)


def test_unpenalised_diagonal_matches_bruteforce():
    X, Y = small_problem(4, 4, 20, seed=30)
    lam_L, lam_T = 0.15, 0.2
    r = tight_solve(X, Y, lam_L, lam_T, penalize_diag=False)
    L_bf, T_bf, f_bf = bf.fista_cggm(X, Y, lam_L, lam_T, iters=60000, penalize_diag=False)
    f_or = bf.cggm_f(r.Lambda, r.Theta, X, Y, lam_L, lam_T, penalize_diag=False)
    assert abs(f_or - f_bf) <= 1e-9 * abs(f_bf)


def test_not_positive_definite_warm_start_raises():
    X, Y = small_problem(4, 3, 20, seed=31)
    bad = np.diag([1.0, -1.0, 1.0])
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.solve(X, Y, 0.1, 0.1, Lambda0=bad)


def test_active_set_strict_threshold():
    """An entry whose gradient equals lam exactly is not active (strict >)."""
    G_L = np.array([[0.5, 0.1], [0.1, 0.5]])
    G_T = np.array([[0.2, -0.2000001]])
    li, lj, ti, tj = oracle.active_sets(G_L, G_T, np.eye(2), np.zeros((1, 2)), 0.1, 0.2)
    assert list(zip(li, lj)) == [(0, 0), (1, 1)]
    assert list(zip(ti, tj)) == [(0, 1)]


# ------------------------------------------------------------------------------------
# sparse SPD solve (Section 4's Sigma columns and P = R Sigma)
# ------------------------------------------------------------------------------------
def test_spd_solve_closed_forms():
    """Diagonal Lambda: X = B / diag.  2 x 2: the adjugate formula.  Chain: the residual
    Lambda X - B vanishes and Sigma = Lambda^-1 is symmetric, with the known sign pattern
    of the inverse of a tridiagonal M-matrix-like chain with positive off-diagonals
    (Sigma_ij (-1)^(i+j) > 0)."""
    rng = np.random.default_rng(0)
    d = rng.uniform(0.5, 2.0, size=9)
    B = rng.standard_normal((9, 4))
    np.testing.assert_allclose(oracle.spd_solve(np.diag(d), B), B / d[:, None], rtol=1e-14)
    a, b, c = 2.0, 0.7, 1.5
    A = np.array([[a, b], [b, c]])
    inv = np.array([[c, -b], [-b, a]]) / (a * c - b * b)
    np.testing.assert_allclose(oracle.spd_solve(A, np.eye(2)), inv, rtol=1e-14)
    Lam = synth.chain_precision(40).toarray()
    S = oracle.spd_solve(Lam, np.eye(40))
    np.testing.assert_allclose(Lam @ S, np.eye(40), atol=1e-12)
    np.testing.assert_allclose(S, S.T, atol=1e-13)
    i, j = np.indices(S.shape)
    assert np.all(S * (-1.0) ** (i + j) > 0)
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.spd_solve(np.array([[1.0, 2.0], [2.0, 1.0]]), np.eye(2))


def test_prediction_at_lambda_zero_is_the_least_squares_fit():
    """Section 2.1's conditional mean at the lambda = 0 optimum: B = -Theta Sigma equals the
    least-squares coefficients S_xx^-1 S_xy, so the predictions are the ordinary
    least-squares fit of Y on X (numpy lstsq, a different algorithm).  A sign flip, a
    transposed Theta or a Lambda in place of Sigma fails it."""
    X, Y = small_problem(6, 4, 60, seed=3)
    r = oracle.solve(X, Y, 0.0, 0.0, tol=1e-13, max_iter=20000)
    Yhat, B = oracle.predict(X, r.Lambda, r.Theta)
    coef, *_ = np.linalg.lstsq(X, Y, rcond=None)
    assert np.max(np.abs(B - coef)) < 1e-7 * np.max(np.abs(coef))
    assert np.max(np.abs(Yhat - X @ coef)) < 1e-7 * np.max(np.abs(Y))
    # scalar case by hand: Lambda = 2, Theta = 3 -> B = -3/2
    Yh, B1 = oracle.predict(np.array([[1.0], [-2.0]]), np.array([[2.0]]), np.array([[3.0]]))
    assert B1[0, 0] == -1.5 and np.allclose(Yh[:, 0], [-1.5, 3.0])
    with pytest.raises(oracle.NotPositiveDefinite):
        oracle.predict(X, -np.eye(4), r.Theta)


def test_full_step_never_meets_sigma_one():
    """Forced line-search exhaustion: the smooth part of Eq. 1 is strictly convex along the
    Newton direction, so at alpha = 1 the objective lies strictly above f + delta (its
    linearisation plus the exact l1 change); with sigma = 1 and a single trial the Armijo
    rule must fail, while the default sigma accepts a step on the same problem."""
    X, Y = small_problem(6, 5, 40, seed=13)
    with pytest.raises(oracle.LineSearchFailed):
        oracle.solve(X, Y, 0.1, 0.1, tol=1e-8, max_iter=3, sigma=1.0, ls_max_trials=1)
    r = oracle.solve(X, Y, 0.1, 0.1, tol=1e-8, max_iter=3)
    assert r.history[0].trials >= 1 and r.history[0].alpha > 0
