"""Model selection over the solver (host orchestration; every solve and objective runs in the
library through the C ABI).

The paper's synthetic experiments (Section 5) choose lambda_Lambda and lambda_Theta so that
the numbers of estimated edges in Lambda and Theta are close to the true ones, and its
edge-recovery study (Fig. 7) compares the estimated support with the true one as n grows.
This module provides those steps:

  edge_counts          off-diagonal edges of Lambda (pairs i < j) and nonzeros of Theta of a
                       solution returned by Context.cggm_solve;
  lambdas_for_edges    lambda_Lambda and lambda_Theta whose solution has (about) given edge
                       counts, by bisection on log lambda with warm starts;
  cross_validate       K-fold cross-validation over a lambda path: each fold's training rows
                       are solved along the path with warm starts, and the held-out rows score
                       each point by the smooth part of Eq. 1 (cggm_objective with zero
                       penalties: the held-out negative log-likelihood up to constants);
  support_f1           precision, recall and F1 of the recovered support against a true one;
  recovery_versus_n    the edge-recovery study: at each sample size n, samples from the true
                       model, penalties matched to the true edge counts, and the F1 of the
                       recovered supports of Lambda and Theta.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np


def edge_counts(result) -> tuple:
    """(edges of Lambda, edges of Theta): pairs i < j with Lambda_ij != 0, and entries with
    Theta_ij != 0, from the coordinate lists of a Context.cggm_solve result."""
    r, c, v = result.Lambda_coo
    e_lam = int(np.count_nonzero((r < c) & (v != 0)))
    e_th = int(np.count_nonzero(result.Theta_coo[2] != 0))
    return e_lam, e_th


@dataclasses.dataclass
class EdgeMatch:
    lam_L: float
    lam_T: float
    edges_L: int
    edges_T: int
    result: object
    solves: int


def lambdas_for_edges(ctx, X, Y, target_L: int, target_T: int, lam_lo: float = 1e-4,
                      lam_hi: float = 1e3, rounds: int = 20, rel_tol: float = 0.05,
                      tol: float = 0.01, opts=None) -> EdgeMatch:
    """lambda_Lambda and lambda_Theta whose solution has about target_L edges in Lambda and
    target_T in Theta (Section 5's choice of the penalties).  Each round solves at the current
    pair (warm-started from the previous solution) and halves, on a log scale, the bracket
    of each penalty whose edge count is off by more than rel_tol: fewer edges than wanted
    means the penalty is too large.  The two counts depend mostly on their own penalty, so
    the brackets are narrowed side by side.  The default bracket, 1e-4 to 1e3, spans the
    gradients' scale for data of unit-order variance (the penalty that empties an active set
    is the largest gradient entry).  Returns the closest pair found."""
    lo = [math.log(lam_lo), math.log(lam_lo)]
    hi = [math.log(lam_hi), math.log(lam_hi)]
    cur = [0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1])]
    best = None
    warm = None
    targets = (max(1, target_L), max(1, target_T))
    for k in range(rounds):
        lam_L, lam_T = math.exp(cur[0]), math.exp(cur[1])
        kw = {} if warm is None else {"warm_Lambda": warm.Lambda_coo, "warm_Theta": warm.Theta_coo}
        res = ctx.cggm_solve(X, Y, lam_L, lam_T, tol=tol, opts=opts, **kw)
        e = edge_counts(res)
        err = max(abs(e[0] - targets[0]) / targets[0], abs(e[1] - targets[1]) / targets[1])
        if best is None or err < best[0]:
            best = (err, EdgeMatch(lam_L, lam_T, e[0], e[1], res, k + 1))
        if err <= rel_tol:
            break
        warm = res
        for d in range(2):
            if abs(e[d] - targets[d]) <= rel_tol * targets[d]:
                continue
            if e[d] < targets[d]:  # too few edges: the penalty is too large
                hi[d] = cur[d]
            else:
                lo[d] = cur[d]
            cur[d] = 0.5 * (lo[d] + hi[d])
    m = best[1]
    m.solves = k + 1
    return m


@dataclasses.dataclass
class CVResult:
    lambdas: list
    loss: np.ndarray      # folds x lambdas: held-out smooth objective
    mean: np.ndarray      # per lambda
    best_lambda: float


def cross_validate(ctx, X, Y, lambdas: Sequence[float], folds: int = 5, seed: int = 0,
                   tol: float = 0.01, opts=None) -> CVResult:
    """K-fold cross-validation over a lambda path (lambda_Lambda = lambda_Theta = lambda):
    rows are split into `folds` folds by a seeded permutation; on each fold's training rows
    the path is solved in the given order with warm starts, and each point is scored on the
    held-out rows by the smooth part of Eq. 1 (zero penalties).  Returns every score, their
    mean per lambda and the lambda of the lowest mean."""
    X = np.asarray(X)
    Y = np.asarray(Y)
    n = X.shape[0]
    perm = np.random.default_rng(seed).permutation(n)
    parts = np.array_split(perm, folds)
    loss = np.empty((folds, len(lambdas)))
    for f, test in enumerate(parts):
        train = np.setdiff1d(perm, test)
        Xtr, Ytr = X[train], Y[train]
        Xte, Yte = X[test], Y[test]
        warm = None
        for k, lam in enumerate(lambdas):
            kw = {} if warm is None else {"warm_Lambda": warm.Lambda_coo, "warm_Theta": warm.Theta_coo}
            res = ctx.cggm_solve(Xtr, Ytr, lam, lam, tol=tol, opts=opts, **kw)
            loss[f, k] = ctx.cggm_objective(Xte, Yte, res.Lambda, res.Theta, 0.0, 0.0)
            warm = res
    mean = loss.mean(axis=0)
    return CVResult(list(lambdas), loss, mean, float(lambdas[int(np.argmin(mean))]))


@dataclasses.dataclass
class SupportScore:
    precision: float
    recall: float
    f1: float
    true_edges: int
    found_edges: int


def support_f1(est, true, threshold: float = 0.0, upper: bool = False) -> SupportScore:
    """Precision, recall and F1 of the estimated support: entries with |est| > threshold
    against the nonzeros of `true` (dense matrices; a sparse `true` with .toarray() is
    accepted).  upper: count only pairs i < j (the edges of a symmetric Lambda)."""
    E = np.asarray(est)
    T = true.toarray() if hasattr(true, "toarray") else np.asarray(true)
    if E.shape != T.shape:
        raise ValueError("est and true differ in shape")
    mask = np.ones(E.shape, dtype=bool)
    if upper:
        mask = np.triu(mask, k=1)
    found = (np.abs(E) > threshold) & mask
    real = (T != 0) & mask
    tp = int(np.count_nonzero(found & real))
    nf, nr = int(np.count_nonzero(found)), int(np.count_nonzero(real))
    precision = tp / nf if nf else (1.0 if nr == 0 else 0.0)
    recall = tp / nr if nr else 1.0
    f1 = 2 * precision * recall / (precision + recall) if precision + recall > 0 else 0.0
    return SupportScore(precision, recall, f1, nr, nf)


@dataclasses.dataclass
class RecoveryPoint:
    n: int
    lam_L: float
    lam_T: float
    lambda_support: SupportScore  # off-diagonal pairs i < j of Lambda
    theta_support: SupportScore
    solves: int


def recovery_versus_n(ctx, sample, Lambda_true, Theta_true, ns: Sequence[int], seed: int = 0,
                      tol: float = 0.01, opts=None, **edge_kw) -> list:
    """The edge-recovery study of Section 5 (Fig. 7): for each sample size n in ns, draw n
    samples of the true model with sample(n, rng) -> (X, Y), choose lambda_Lambda and
    lambda_Theta whose solution has the true numbers of edges (lambdas_for_edges, the
    paper's choice of penalties), and score the recovered supports of Lambda (pairs i < j)
    and Theta against the true ones (support_f1).  Lambda_true and Theta_true are dense or
    sparse (with .toarray()); edge_kw passes the bracket and rounds to lambdas_for_edges.
    One seeded generator draws every n's samples in turn."""
    Lt = Lambda_true.toarray() if hasattr(Lambda_true, "toarray") else np.asarray(Lambda_true)
    Tt = Theta_true.toarray() if hasattr(Theta_true, "toarray") else np.asarray(Theta_true)
    target_L = int(np.count_nonzero(np.triu(Lt, 1)))
    target_T = int(np.count_nonzero(Tt))
    rng = np.random.default_rng(seed)
    points = []
    for n in ns:
        X, Y = sample(int(n), rng)
        m = lambdas_for_edges(ctx, X, Y, target_L, target_T, tol=tol, opts=opts, **edge_kw)
        points.append(RecoveryPoint(int(n), m.lam_L, m.lam_T,
                                    support_f1(m.result.Lambda, Lt, upper=True),
                                    support_f1(m.result.Theta, Tt), m.solves))
    return points
