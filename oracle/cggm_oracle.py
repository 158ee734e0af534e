"""Double-precision CPU oracle of the alternating Newton coordinate-descent solver.

TEST INFRASTRUCTURE (see the package docstring).  Dense numpy linear algebra serves as
library steps (matrix products, Cholesky); the two coordinate-descent passes are the
plain C loops of ``sweeps.c``.  Every function names the passage it follows.

Readings of the paper taken here (each is stated where it is used):
  * the curvature a of a Lambda coordinate is the exact second derivative of the
    quadratic model, S_ij^2 + S_ii S_jj + S_ii P_jj + S_jj P_ii + 2 S_ij P_ij, and the
    Theta curvature is 2 Sigma_jj (S_xx)_ii (Appendix A.1 prints other values);
  * ||Lambda||_1 includes the diagonal unless ``penalize_diag`` is False (Eq. 1 says
    "elementwise");
  * Armijo: alpha = 1, beta, beta^2, ... with sigma = 1e-3, beta = 0.5, at most 50 trials,
    decrease measured against delta = tr(G_Lambda D) + lam (||Lambda+D||_1 - ||Lambda||_1);
  * coordinates are visited row-major: (i, j) with i <= j for Lambda, all (i, j) for
    Theta, ascending;
  * the Theta pass uses Sigma of the accepted Lambda;
  * the stopping rule sums the minimum-norm subgradient over every entry of Lambda
    (both triangles) and Theta, against tol (||Lambda||_1 + ||Theta||_1) over the same
    entries;
  * an entry is active when |gradient| > lam strictly, or the parameter is nonzero.
"""
from __future__ import annotations

import ctypes
import dataclasses
import time
from typing import Optional

import numpy as np

from . import build as _build


class OracleError(RuntimeError):
    pass


class NotPositiveDefinite(OracleError):
    pass


class LineSearchFailed(OracleError):
    pass


_LIBS = {}


def _lib(mutant: bool = False):
    if mutant not in _LIBS:
        lib = ctypes.CDLL(_build.build(mutant=mutant))
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.c_int64
        lib.oracle_lambda_sweep.argtypes = [i64, dp, dp, dp, dp, i64, ip, ip,
                                            ctypes.c_double, ctypes.c_double, dp, dp]
        lib.oracle_lambda_sweep.restype = None
        lib.oracle_theta_sweep.argtypes = [i64, i64, dp, dp, dp, i64, ip, ip,
                                           ctypes.c_double, dp, dp]
        lib.oracle_theta_sweep.restype = None
        _LIBS[mutant] = lib
    return _LIBS[mutant]


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def soft_threshold(w, r):
    """S_r(w) = sign(w) max(|w| - r, 0) (Appendix A.1)."""
    return np.sign(w) * np.maximum(np.abs(w) - r, 0.0)


def covariances(X: np.ndarray, Y: np.ndarray):
    """S_xx = X^T X / n, S_xy = X^T Y / n, S_yy = Y^T Y / n (Section 2.1); no centring."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n = X.shape[0]
    return X.T @ X / n, X.T @ Y / n, Y.T @ Y / n


def _chol(Lam: np.ndarray) -> np.ndarray:
    try:
        return np.linalg.cholesky(Lam)
    except np.linalg.LinAlgError as e:
        raise NotPositiveDefinite(str(e)) from None


def spd_solve(Lam: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = Lambda^-1 B for a symmetric positive definite Lambda (dense).  Section 4 computes
    columns of Sigma = Lambda^-1 (B = identity columns) and P = R Sigma (B = R^T) this way by
    conjugate gradient on the sparse Lambda; the oracle is the definition, with a Cholesky
    factorisation and two triangular solves as library steps."""
    L = _chol(Lam)
    Z = np.linalg.solve(L, B)
    return np.linalg.solve(L.T, Z)


def _l1(A: np.ndarray, penalize_diag: bool = True) -> float:
    s = float(np.abs(A).sum())
    if not penalize_diag and A.shape[0] == A.shape[1]:
        s -= float(np.abs(np.diag(A)).sum())
    return s


def smooth_objective(Lam, Theta, Sxx, Sxy, Syy) -> float:
    """g(Lambda, Theta) = -log|Lambda| + tr(S_yy Lambda + 2 S_xy^T Theta
    + Lambda^-1 Theta^T S_xx Theta)  (Eq. 1).  Raises NotPositiveDefinite."""
    L = _chol(Lam)
    logdet = 2.0 * float(np.log(np.diag(L)).sum())
    A = Theta.T @ Sxx @ Theta
    # tr(Lambda^-1 A) = ||L^-1 A^(1/2)||^2 in exact arithmetic; here solve L W = A, L^T Z = W
    Z = np.linalg.solve(L.T, np.linalg.solve(L, A))
    return -logdet + float(np.sum(Syy * Lam)) + 2.0 * float(np.sum(Sxy * Theta)) + float(np.trace(Z))


def objective(Lam, Theta, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag=True) -> float:
    """f = g + lam_L ||Lambda||_1 + lam_T ||Theta||_1 (Eq. 1)."""
    return smooth_objective(Lam, Theta, Sxx, Sxy, Syy) + lam_L * _l1(Lam, penalize_diag) \
        + lam_T * _l1(Theta)


def gradients(Lam, Theta, Sxx, Sxy, Syy, Sigma: Optional[np.ndarray] = None):
    """Eq. 3: grad_Lambda g = S_yy - Sigma - Psi, grad_Theta g = 2 S_xy + 2 Gamma, with
    Sigma = Lambda^-1, Psi = Sigma Theta^T S_xx Theta Sigma, Gamma = S_xx Theta Sigma.
    Returns (G_Lambda, G_Theta, Sigma, Psi)."""
    if Sigma is None:
        L = _chol(Lam)
        Linv = np.linalg.solve(L, np.eye(L.shape[0]))
        Sigma = Linv.T @ Linv
    V = Theta @ Sigma
    Psi = V.T @ Sxx @ V
    G_L = Syy - Sigma - Psi
    G_T = 2.0 * Sxy + 2.0 * (Sxx @ V)
    return G_L, G_T, Sigma, Psi


def min_norm_subgradient(G: np.ndarray, P: np.ndarray, lam, lam_diag=None) -> np.ndarray:
    """Entry-wise minimum-norm subgradient of g + lam ||.||_1 at P given grad g = G
    (the stopping quantity of Section 5.1): G + lam sign(P) where P != 0, and
    sign(G) max(|G| - lam, 0) where P = 0.  ``lam_diag`` overrides lam on the diagonal."""
    lam_m = np.full(G.shape, float(lam))
    if lam_diag is not None:
        np.fill_diagonal(lam_m, float(lam_diag))
    nz = P != 0
    return np.where(nz, G + lam_m * np.sign(P), np.sign(G) * np.maximum(np.abs(G) - lam_m, 0.0))


def active_sets(G_L, G_T, Lam, Theta, lam_L, lam_T, penalize_diag=True):
    """S_Lambda, S_Theta of Section 2.2: |grad| > lam (strict) or parameter != 0.
    Lambda entries are listed for i <= j only (the direction is symmetric).  Both
    lists are row-major ascending.  Returns (li, lj, ti, tj) as int32 arrays."""
    q = Lam.shape[0]
    thr = np.full((q, q), float(lam_L))
    if not penalize_diag:
        # with no penalty on the diagonal every diagonal entry is active: |G| > 0 or
        # Lambda_ii != 0, and Lambda_ii > 0 always holds for positive definite Lambda
        np.fill_diagonal(thr, -1.0)
    actL = (np.abs(G_L) > thr) | (Lam != 0)
    actL = np.triu(actL)
    li, lj = np.nonzero(actL)
    actT = (np.abs(G_T) > lam_T) | (Theta != 0)
    ti, tj = np.nonzero(actT)
    return (li.astype(np.int32), lj.astype(np.int32), ti.astype(np.int32), tj.astype(np.int32))


def lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, lam_L, penalize_diag=True, mutant=False):
    """One CD pass for the Newton direction D (Section 3.1, Eq. 7; C loop in sweeps.c)."""
    q = Lam.shape[0]
    D = np.zeros((q, q))
    Ut = np.zeros((q, q))
    args = [np.ascontiguousarray(a, dtype=np.float64) for a in (Sigma, Psi, Syy, Lam)]
    li = np.ascontiguousarray(li, dtype=np.int32)
    lj = np.ascontiguousarray(lj, dtype=np.int32)
    _lib(mutant).oracle_lambda_sweep(q, *map(_dp, args), li.size, _ip(li), _ip(lj),
                                     float(lam_L), float(lam_L) if penalize_diag else 0.0,
                                     _dp(D), _dp(Ut))
    return D


def theta_sweep(Sxx, Sxy, Sigma, Theta, ti, tj, lam_T, mutant=False):
    """One CD pass over the active entries of Theta (Section 3.2, Eq. 8; C loop)."""
    p, q = Theta.shape
    Th = np.array(Theta, dtype=np.float64, order="C", copy=True)
    Vt = np.ascontiguousarray((Th @ Sigma).T)
    Sxx = np.ascontiguousarray(Sxx, dtype=np.float64)
    Sxy = np.ascontiguousarray(Sxy, dtype=np.float64)
    Sigma = np.ascontiguousarray(Sigma, dtype=np.float64)
    ti = np.ascontiguousarray(ti, dtype=np.int32)
    tj = np.ascontiguousarray(tj, dtype=np.int32)
    _lib(mutant).oracle_theta_sweep(p, q, _dp(Sxx), _dp(Sxy), _dp(Sigma), ti.size, _ip(ti),
                                    _ip(tj), float(lam_T), _dp(Th), _dp(Vt))
    return Th


def line_search(Lam, D, Theta, Sxx, Sxy, Syy, G_L, f0, lam_L, lam_T, penalize_diag=True,
                sigma=1e-3, beta=0.5, max_trials=50):
    """Armijo rule on Lambda + alpha D (Algorithm 1, Section 2.2): the largest alpha in
    {1, beta, beta^2, ...} with Lambda + alpha D positive definite and
    f(Lambda + alpha D, Theta) <= f + sigma alpha delta,
    delta = tr(G_Lambda D) + lam_L (||Lambda + D||_1 - ||Lambda||_1).
    Returns (alpha, f_alpha, trials)."""
    delta = float(np.sum(G_L * D)) + lam_L * (_l1(Lam + D, penalize_diag) - _l1(Lam, penalize_diag))
    alpha = 1.0
    for k in range(1, max_trials + 1):
        La = Lam + alpha * D
        try:
            fa = objective(La, Theta, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag)
        except NotPositiveDefinite:
            fa = None
        if fa is not None and fa <= f0 + sigma * alpha * delta:
            return alpha, fa, k
        alpha *= beta
    raise LineSearchFailed(f"no step after {max_trials} trials (delta={delta:g})")


@dataclasses.dataclass
class IterRecord:
    it: int
    f: float                 # objective at the start of the iteration
    subgrad: float           # ||grad^S||_1 at the start of the iteration
    l1_norm: float           # ||Lambda||_1 + ||Theta||_1 (all entries)
    m_L: int
    m_T: int
    alpha: float = float("nan")
    trials: int = 0
    seconds: float = 0.0


@dataclasses.dataclass
class SolveResult:
    Lambda: np.ndarray
    Theta: np.ndarray
    f: float
    iterations: int
    converged: bool
    history: list


def solve(X, Y, lam_L, lam_T, tol=0.01, max_iter=100, Lambda0=None, Theta0=None,
          penalize_diag=True, sigma=1e-3, beta=0.5, ls_max_trials=50, mutant=False,
          callback=None, cov=None) -> SolveResult:
    """Alternating Newton coordinate descent (Algorithm 1).

    Theta <- 0, Lambda <- I (or the warm start); each iteration: Sigma, Psi and the
    gradients (Eq. 3); stop when the minimum-norm subgradient ratio falls below tol;
    active sets; one CD pass for D (Eq. 7); Armijo step on Lambda; one CD pass on
    Theta with the new Sigma (Eq. 8)."""
    Sxx, Sxy, Syy = cov if cov is not None else covariances(X, Y)
    p, q = Sxy.shape
    Lam = np.eye(q) if Lambda0 is None else np.array(Lambda0, dtype=np.float64, copy=True)
    Th = np.zeros((p, q)) if Theta0 is None else np.array(Theta0, dtype=np.float64, copy=True)
    lam_diag = lam_L if penalize_diag else 0.0
    hist = []
    converged = False
    Sigma = None
    f = objective(Lam, Th, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag)
    for it in range(max_iter):
        t0 = time.perf_counter()
        G_L, G_T, Sigma, Psi = gradients(Lam, Th, Sxx, Sxy, Syy, Sigma)
        gs = float(np.abs(min_norm_subgradient(G_L, Lam, lam_L, lam_diag)).sum()
                   + np.abs(min_norm_subgradient(G_T, Th, lam_T)).sum())
        nrm = _l1(Lam) + _l1(Th)
        li, lj, ti, tj = active_sets(G_L, G_T, Lam, Th, lam_L, lam_T, penalize_diag)
        rec = IterRecord(it=it, f=f, subgrad=gs, l1_norm=nrm, m_L=int(li.size), m_T=int(ti.size))
        if gs < tol * nrm:
            converged = True
            hist.append(rec)
            if callback:
                callback(rec, Lam, Th)
            break
        D = lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, lam_L, penalize_diag, mutant=mutant)
        alpha, f_ls, trials = line_search(Lam, D, Th, Sxx, Sxy, Syy, G_L, f, lam_L, lam_T,
                                          penalize_diag, sigma, beta, ls_max_trials)
        Lam = Lam + alpha * D
        L = _chol(Lam)
        Linv = np.linalg.solve(L, np.eye(q))
        Sigma = Linv.T @ Linv
        Th = theta_sweep(Sxx, Sxy, Sigma, Th, ti, tj, lam_T, mutant=mutant)
        f = objective(Lam, Th, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag)
        rec.alpha, rec.trials, rec.seconds = alpha, trials, time.perf_counter() - t0
        hist.append(rec)
        if callback:
            callback(rec, Lam, Th)
    return SolveResult(Lambda=Lam, Theta=Th, f=f, iterations=len(hist), converged=converged,
                       history=hist)


def predict(X, Lam, Theta):
    """Conditional mean of the outputs given the inputs (Section 2.1): y | x has mean
    -Lambda^-1 Theta^T x, so the n rows of X predict Yhat = X B with the regression
    coefficients B = -Theta Sigma, Sigma = Lambda^-1.  Returns (Yhat, B)."""
    Lam = np.asarray(Lam, dtype=np.float64)
    _chol(Lam)  # positive definite, or NotPositiveDefinite
    B = -np.asarray(Theta, dtype=np.float64) @ np.linalg.inv(Lam)
    return np.asarray(X, dtype=np.float64) @ B, B
