"""Alternating Newton block coordinate descent (Algorithm 2, Section 4): oracle form.

TEST INFRASTRUCTURE (see the package docstring).  Plain numpy, double precision, loops in
Python: for small cases only.

Section 4 runs the two coordinate passes of Algorithm 1 in an order set by a partition of
the q output columns into blocks C_1..C_k, so that only a few columns of the large
matrices are held at a time.  What is held here is what the section holds:

  * Lambda pass (Section 4.1): for block z, the columns Sigma_{C_z} (solves with
    Lambda), Psi_{C_z} = P^T P_{C_z} / n with P = X Theta Sigma, and U_{C_z} = D Sigma_{C_z};
    for an off-diagonal block (C_z, C_r) with active entries, the same three for C_r
    (a cache miss).  After a step on (a, b), rows a and b of U grow at the held columns
    only; U's other columns are formed again from D when their block is loaded.
  * Theta pass (Section 4.2): for block r, Sigma_{C_r} and V_{C_r} = Theta Sigma_{C_r};
    for each row i with active entries in (i, C_r), the row (S_xx)_{i,K} = X_i^T X_K / n
    over the rows K of Theta that hold an active entry (a cache miss); no p x p S_xx.

Readings taken here (the paper does not fix them):
  B1  each symmetric Lambda coordinate is stepped once per pass, in the block pair
      (z, r), z <= r, of its two indices' blocks;
  B2  inside a block pair the coordinates run over a in C_z, then b in C_r, both by
      ascending column index (a <= b in a diagonal block); Theta blocks run over rows i
      ascending, then j in C_r ascending;
  B3  K is the set of rows of Theta with an active entry (rows outside it are zero in
      Theta and in V, so their S_xx entries do not enter any dot product);
  B4  Sigma_{C_z} is formed for every block z (Algorithm 2 does so unconditionally);
      C_r is loaded for z != r only when (C_z, C_r) holds an active coordinate.

Since every step is the exact one-dimensional minimiser of Appendix A.1 on the current
iterate, each blocked pass equals the sequential pass of Algorithm 1 run over the same
coordinates in the blocked order (up to the order of floating-point sums).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np

from .cggm_oracle import (
    IterRecord,
    SolveResult,
    _l1,
    active_sets,
    covariances,
    gradients,
    line_search,
    min_norm_subgradient,
    objective,
    spd_solve,
)


def block_lists(block) -> list:
    """The column sets C_1..C_k of a partition given as one block id per column (ids
    0..k-1, every id used), each as ascending column indices."""
    block = np.asarray(block, dtype=np.int64)
    k = int(block.max()) + 1 if block.size else 0
    C = [np.flatnonzero(block == z) for z in range(k)]
    if any(c.size == 0 for c in C):
        raise ValueError("block ids must be 0..k-1 with no empty block")
    return C


def lambda_block_order(li, lj, block) -> np.ndarray:
    """Positions of the active Lambda coordinates (i <= j) in the visiting order of the
    blocked pass (readings B1, B2): by block pair (z, r), z <= r, then a in C_z, then b
    in C_r, where {a, b} = {i, j} with a in the lower-numbered block."""
    li = np.asarray(li, dtype=np.int64)
    lj = np.asarray(lj, dtype=np.int64)
    block = np.asarray(block, dtype=np.int64)
    bi, bj = block[li], block[lj]
    swap = bi > bj
    a = np.where(swap, lj, li)
    b = np.where(swap, li, lj)
    z = np.minimum(bi, bj)
    r = np.maximum(bi, bj)
    return np.lexsort((b, a, r, z))


def theta_block_order(ti, tj, block) -> np.ndarray:
    """Positions of the active Theta coordinates in the visiting order of the blocked pass
    (reading B2): by the block r of j, then row i, then j."""
    ti = np.asarray(ti, dtype=np.int64)
    tj = np.asarray(tj, dtype=np.int64)
    r = np.asarray(block, dtype=np.int64)[tj]
    return np.lexsort((tj, ti, r))


def _soft(w: float, r: float) -> float:
    if w > r:
        return w - r
    if w < -r:
        return w + r
    return 0.0


@dataclasses.dataclass
class BlockStats:
    columns: int = 0      # columns of Sigma (and of Psi, U, for Lambda) formed
    misses: int = 0       # Lambda: off-diagonal blocks loaded; Theta: rows (S_xx)_i formed
    blocks_visited: int = 0


def lambda_sweep_blocked(Lam, P, Syy, li, lj, block, lam_L, penalize_diag=True):
    """One blocked CD pass for the Newton direction D (Algorithm 2, Section 4.1).

    Lam: Lambda (q x q); P = X Theta Sigma (n x q); Syy (q x q); li, lj the active
    coordinates (i <= j, any order: they are visited in the blocked order); block: one
    block id per column.  Returns (D, BlockStats)."""
    Lam = np.asarray(Lam, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    q = Lam.shape[0]
    n = P.shape[0]
    lam_diag = float(lam_L) if penalize_diag else 0.0
    C = block_lists(block)
    block = np.asarray(block, dtype=np.int64)
    li = np.asarray(li, dtype=np.int64)
    lj = np.asarray(lj, dtype=np.int64)
    order = lambda_block_order(li, lj, block)
    groups: dict = {}
    for t in order:
        i, j = int(li[t]), int(lj[t])
        a, b = (i, j) if block[i] <= block[j] else (j, i)
        groups.setdefault((int(block[a]), int(block[b])), []).append((a, b))
    D = np.zeros((q, q))
    st = BlockStats()
    eye = np.eye(q)

    def load(cols):
        # Sigma_C by solves with Lambda; Psi_C = P^T P_C / n; U_C = D Sigma_C
        S = spd_solve(Lam, eye[:, cols])
        Ps = P.T @ P[:, cols] / n
        U = D @ S
        st.columns += cols.size
        return S, Ps, U, {int(c): t for t, c in enumerate(cols)}

    for z in range(len(C)):
        Sz, Pz, Uz, pz = load(C[z])
        for r in range(z, len(C)):
            coords = groups.get((z, r))
            if not coords:
                continue
            st.blocks_visited += 1
            if r == z:
                Sr, Pr, Ur, pr = Sz, Pz, Uz, pz
            else:
                Sr, Pr, Ur, pr = load(C[r])
                st.misses += 1
            for a, b in coords:
                sa, sb = Sz[:, pz[a]], Sr[:, pr[b]]       # columns a, b of Sigma
                pa, pb = Pz[:, pz[a]], Pr[:, pr[b]]       # columns a, b of Psi
                ua, ub = Uz[:, pz[a]], Ur[:, pr[b]]       # columns a, b of U = D Sigma
                s_aa, s_bb, s_ab = sa[a], sb[b], sa[b]
                p_aa, p_bb, p_ab = pa[a], pb[b], pa[b]
                sds = float(sa @ ub)                     # (Sigma D Sigma)_ab
                pds_ab = float(pa @ ub)                  # (Psi D Sigma)_ab
                if a != b:
                    pds_ba = float(pb @ ua)              # (Psi D Sigma)_ba
                    curv = s_ab * s_ab + s_aa * s_bb + s_aa * p_bb + s_bb * p_aa + 2.0 * s_ab * p_ab
                    lin = Syy[a, b] - s_ab - p_ab + sds + pds_ab + pds_ba
                    lam = float(lam_L)
                else:
                    curv = s_aa * s_aa + 2.0 * s_aa * p_aa
                    lin = Syy[a, a] - s_aa - p_aa + sds + 2.0 * pds_ab
                    lam = lam_diag
                c = Lam[a, b] + D[a, b]
                mu = -c + _soft(c - lin / curv, lam / curv)
                if mu == 0.0:
                    continue
                D[a, b] += mu
                if a != b:
                    D[b, a] += mu
                # U_a += mu Sigma_b, U_b += mu Sigma_a at the held columns C_z (and C_r)
                Uz[a, :] += mu * Sz[b, :]
                if a != b:
                    Uz[b, :] += mu * Sz[a, :]
                if r != z:
                    Ur[a, :] += mu * Sr[b, :]
                    if a != b:
                        Ur[b, :] += mu * Sr[a, :]
    return D, st


def theta_sweep_blocked(X, Sxy, Lam, Theta, ti, tj, block, lam_T):
    """One blocked CD pass over the active entries of Theta (Algorithm 2, Section 4.2).

    X (n x p); Sxy (p x q); Lam: Lambda (its columns Sigma_{C_r} come from solves);
    Theta (p x q, not modified); ti, tj the active coordinates (any order); block: one
    block id per output column.  Returns (Theta_new, BlockStats)."""
    X = np.asarray(X, dtype=np.float64)
    Lam = np.asarray(Lam, dtype=np.float64)
    n, p = X.shape
    q = Lam.shape[0]
    Th = np.array(Theta, dtype=np.float64, copy=True)
    C = block_lists(block)
    block = np.asarray(block, dtype=np.int64)
    ti = np.asarray(ti, dtype=np.int64)
    tj = np.asarray(tj, dtype=np.int64)
    K = np.unique(ti)                                   # reading B3
    rows_by_block: list = [dict() for _ in C]
    for t in theta_block_order(ti, tj, block):
        i, j = int(ti[t]), int(tj[t])
        rows_by_block[int(block[j])].setdefault(i, []).append(j)
    st = BlockStats()
    eye = np.eye(q)
    for r, cols in enumerate(C):
        Sr = spd_solve(Lam, eye[:, cols])               # Sigma_{C_r}, q x |C_r|
        st.columns += cols.size
        pr = {int(c): t for t, c in enumerate(cols)}
        V = Th @ Sr                                     # V_{C_r} = Theta Sigma_{C_r}
        for i in sorted(rows_by_block[r]):
            st.blocks_visited += 1
            sxx_iK = X[:, i] @ X[:, K] / n              # (S_xx)_{i,K}: the cache miss
            sxx_ii = float(X[:, i] @ X[:, i]) / n
            st.misses += 1
            for j in rows_by_block[r][i]:
                c = Th[i, j]
                if sxx_ii == 0.0:
                    mu = -c
                else:
                    curv = 2.0 * Sr[j, pr[j]] * sxx_ii
                    lin = 2.0 * Sxy[i, j] + 2.0 * float(sxx_iK @ V[K, pr[j]])
                    mu = -c + _soft(c - lin / curv, float(lam_T) / curv)
                if mu == 0.0:
                    continue
                Th[i, j] += mu
                V[i, :] += mu * Sr[j, :]                # V_i += mu Sigma_{j, C_r}
    return Th, st


def contiguous_partition(q: int, max_block: int) -> np.ndarray:
    """Columns 0..q-1 cut into consecutive blocks of at most ``max_block`` columns."""
    return (np.arange(q) // max(1, int(max_block))).astype(np.int64)


def solve_blocked(X, Y, lam_L, lam_T, max_block: int, tol=0.01, max_iter=100,
                  partition: Optional[Callable] = None, penalize_diag=True, sigma=1e-3,
                  beta=0.5, ls_max_trials=50) -> SolveResult:
    """Alternating Newton block coordinate descent (Algorithm 2).

    Each iteration: gradients and the stopping rule as in Algorithm 1; active sets; a
    partition of the columns of Lambda (``partition('lambda', q, li, lj, max_block)``) and
    of Theta (``partition('theta', q, ti, tj, max_block)``), contiguous blocks when none is
    given; the blocked Lambda pass; the Armijo step; the blocked Theta pass with the new
    Lambda.  Sigma, Psi and S_xx are used whole only for the gradients, the stopping rule
    and the line search, which Section 4 leaves to other means (a sparse Cholesky, solves)
    and which are not what the blocked passes change."""
    X = np.asarray(X, dtype=np.float64)
    Sxx, Sxy, Syy = covariances(X, Y)
    p, q = Sxy.shape
    part = partition or (lambda kind, qq, ii, jj, mb: contiguous_partition(qq, mb))
    Lam = np.eye(q)
    Th = np.zeros((p, q))
    lam_diag = lam_L if penalize_diag else 0.0
    hist = []
    converged = False
    f = objective(Lam, Th, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag)
    for it in range(max_iter):
        G_L, G_T, Sigma, Psi = gradients(Lam, Th, Sxx, Sxy, Syy)
        gs = float(np.abs(min_norm_subgradient(G_L, Lam, lam_L, lam_diag)).sum()
                   + np.abs(min_norm_subgradient(G_T, Th, lam_T)).sum())
        nrm = _l1(Lam) + _l1(Th)
        li, lj, ti, tj = active_sets(G_L, G_T, Lam, Th, lam_L, lam_T, penalize_diag)
        rec = IterRecord(it=it, f=f, subgrad=gs, l1_norm=nrm, m_L=int(li.size), m_T=int(ti.size))
        if gs < tol * nrm:
            converged = True
            hist.append(rec)
            break
        P = spd_solve(Lam, (X @ Th).T).T                # P = X Theta Sigma
        D, _ = lambda_sweep_blocked(Lam, P, Syy, li, lj, part("lambda", q, li, lj, max_block),
                                    lam_L, penalize_diag)
        alpha, _, trials = line_search(Lam, D, Th, Sxx, Sxy, Syy, G_L, f, lam_L, lam_T,
                                       penalize_diag, sigma, beta, ls_max_trials)
        Lam = Lam + alpha * D
        Th, _ = theta_sweep_blocked(X, Sxy, Lam, Th, ti, tj, part("theta", q, ti, tj, max_block),
                                    lam_T)
        f = objective(Lam, Th, Sxx, Sxy, Syy, lam_L, lam_T, penalize_diag)
        rec.alpha, rec.trials = alpha, trials
        hist.append(rec)
    return SolveResult(Lambda=Lam, Theta=Th, f=f, iterations=len(hist), converged=converged,
                       history=hist)
