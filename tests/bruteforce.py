"""Independent brute-force solvers used to pin the oracle.

Nothing here shares arithmetic with ``oracle``: gradients come from torch autograd of
Eq. 1 written directly (log-determinant and traces), and the solvers are textbook
proximal-gradient methods, not coordinate descent.
"""
from __future__ import annotations

import numpy as np
import torch


def _smooth_torch(Lam, Th, Sxx, Sxy, Syy):
    # Eq. 1 smooth part, as written in the paper
    return (-torch.logdet(Lam) + torch.trace(Syy @ Lam) + 2.0 * torch.trace(Sxy.T @ Th)
            + torch.trace(torch.linalg.solve(Lam, Th.T @ Sxx @ Th)))


def cggm_f(Lam, Th, X, Y, lam_L, lam_T, penalize_diag=True):
    """Objective of Eq. 1 from the raw data, in float64 torch (no shared code)."""
    X = torch.as_tensor(X, dtype=torch.float64)
    Y = torch.as_tensor(Y, dtype=torch.float64)
    n = X.shape[0]
    Sxx, Sxy, Syy = X.T @ X / n, X.T @ Y / n, Y.T @ Y / n
    L = torch.as_tensor(Lam, dtype=torch.float64)
    T = torch.as_tensor(Th, dtype=torch.float64)
    pen = L.abs().sum() - (0.0 if penalize_diag else L.diagonal().abs().sum())
    return float(_smooth_torch(L, T, Sxx, Sxy, Syy) + lam_L * pen + lam_T * T.abs().sum())


def fista_cggm(X, Y, lam_L, lam_T, iters=20000, penalize_diag=True, tol=1e-14):
    """Accelerated proximal gradient (FISTA with backtracking and a positive-definite
    safeguard) on (Lambda, Theta) jointly, for tiny problems.  Gradients by autograd."""
    X = torch.as_tensor(X, dtype=torch.float64)
    Y = torch.as_tensor(Y, dtype=torch.float64)
    n, p = X.shape
    q = Y.shape[1]
    Sxx, Sxy, Syy = X.T @ X / n, X.T @ Y / n, Y.T @ Y / n
    lamL = torch.full((q, q), float(lam_L), dtype=torch.float64)
    if not penalize_diag:
        lamL.fill_diagonal_(0.0)

    def smooth(L, T):
        return _smooth_torch(L, T, Sxx, Sxy, Syy)

    def grad(L, T):
        L = L.clone().requires_grad_(True)
        T = T.clone().requires_grad_(True)
        v = smooth(L, T)
        gL, gT = torch.autograd.grad(v, (L, T))
        return v.detach(), 0.5 * (gL + gL.T), gT

    def prox(L, T, step):
        L2 = torch.sign(L) * torch.clamp(L.abs() - step * lamL, min=0.0)
        T2 = torch.sign(T) * torch.clamp(T.abs() - step * lam_T, min=0.0)
        return 0.5 * (L2 + L2.T), T2

    def pd(L):
        try:
            torch.linalg.cholesky(L)
            return True
        except RuntimeError:
            return False

    def F(L, T):
        return float(smooth(L, T) + (lamL * L.abs()).sum() + lam_T * T.abs().sum())

    L = torch.eye(q, dtype=torch.float64)
    T = torch.zeros(p, q, dtype=torch.float64)
    Lx, Tx = L.clone(), T.clone()
    t = 1.0
    step = 1.0
    fprev = F(L, T)
    for _ in range(iters):
        v, gL, gT = grad(Lx, Tx)
        while True:
            Ln, Tn = prox(Lx - step * gL, Tx - step * gT, step)
            if pd(Ln):
                dL, dT = Ln - Lx, Tn - Tx
                vn = smooth(Ln, Tn)
                quad = v + (gL * dL).sum() + (gT * dT).sum() + \
                    ((dL * dL).sum() + (dT * dT).sum()) / (2 * step)
                if vn <= quad + 1e-15 * abs(float(v)):
                    break
            step *= 0.5
            if step < 1e-20:
                raise RuntimeError("FISTA step underflow")
        fn = F(Ln, Tn)
        if fn > fprev:  # restart momentum (monotone variant)
            t = 1.0
            Lx, Tx = L.clone(), T.clone()
            continue
        t_next = 0.5 * (1 + (1 + 4 * t * t) ** 0.5)
        Lx = Ln + (t - 1) / t_next * (Ln - L)
        Tx = Tn + (t - 1) / t_next * (Tn - T)
        if not pd(Lx):
            Lx, Tx = Ln.clone(), Tn.clone()
            t_next = 1.0
        converged = abs(fprev - fn) <= tol * max(1.0, abs(fn))
        L, T, t, fprev = Ln, Tn, t_next, fn
        step *= 1.5
        if converged:
            break
    return L.numpy(), T.numpy(), fprev


def lasso_cd(X, y, alpha, iters=100000, tol=1e-15):
    """Textbook cyclic coordinate-descent Lasso: min (1/n)||y - Xw||^2 + alpha ||w||_1."""
    n, p = X.shape
    w = np.zeros(p)
    r = y.astype(np.float64).copy()
    col = (X * X).sum(axis=0) / n
    for _ in range(iters):
        wmax = 0.0
        for k in range(p):
            if col[k] == 0:
                continue
            rho = X[:, k] @ r / n + col[k] * w[k]
            wk = np.sign(rho) * max(abs(rho) - alpha / 2, 0.0) / col[k]
            if wk != w[k]:
                r -= X[:, k] * (wk - w[k])
                wmax = max(wmax, abs(wk - w[k]))
                w[k] = wk
        if wmax < tol:
            break
    return w
