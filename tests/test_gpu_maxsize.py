"""The largest sizes of the configured workloads (q = 20000 for Lambda, p = 40000 for Theta),
through the coordinate passes in the mixed path's launch configuration, over bounded parts of
their active sets that include the last rows (the largest indices), against the oracle's
sequential passes on the same coordinates (needs a GPU; about 25 GB of host memory)."""
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


def sym_noise(q, scale, rng):
    A = rng.standard_normal((q, q)) * scale
    A += A.T
    return A


def test_lambda_pass_at_q_20000(ctx):
    q = 20000
    rng = np.random.default_rng(7)
    Sigma = sym_noise(q, 1e-3, rng)
    Sigma[np.diag_indices(q)] += 2.0
    Psi = sym_noise(q, 1e-4, rng)
    Psi[np.diag_indices(q)] += 0.1
    Syy = Sigma.copy()
    Syy[np.diag_indices(q)] += 0.3
    Lam = np.eye(q)
    # coordinates: the first row and the last two rows of the upper triangle (largest indices)
    first = [(0, j) for j in range(0, 6000)]
    last = [(i, j) for i in (q - 60, q - 2, q - 1) for j in range(i, q)]
    li = np.array([a for a, _ in first + last], dtype=np.int32)
    lj = np.array([b for _, b in first + last], dtype=np.int32)
    D_ref = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.01)
    D = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.01, precision=cg.CGGM_MIXED)
    assert np.abs(D_ref[q - 1, q - 1]) > 0 and np.abs(D_ref).max() > 0
    assert rel(D, D_ref) < 2e-4


def covariances_in_row_blocks(X, Y, block=5000):
    """S_xx = X^T X / n and S_xy = X^T Y / n (Section 2.1), S_xx formed a block of rows at a
    time: a single 40000 x 40000 product is more than the host BLAS takes in one call."""
    n, p = X.shape
    Sxx = np.empty((p, p))
    for r0 in range(0, p, block):
        Sxx[r0:r0 + block] = X[:, r0:r0 + block].T @ X / n
    return Sxx, X.T @ Y / n


def test_theta_pass_at_p_40000(ctx):
    p, q, n = 40000, 64, 200
    pr = synth.make_problem(p, q, n, x_kind="genotype", seed=8, theta_nnz=3)
    Sxx, Sxy = covariances_in_row_blocks(pr.X, pr.Y)
    Th = 0.5 * pr.Theta_true.toarray()
    Sigma = np.linalg.inv(pr.Lambda_true.toarray())
    rows = np.array([0, 1, 2, p - 5, p - 2, p - 1])
    ti = np.repeat(rows, q).astype(np.int32)
    tj = np.tile(np.arange(q), rows.size).astype(np.int32)
    T_ref = oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti, tj, 0.02)
    T = ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, ti, tj, 0.02, precision=cg.CGGM_MIXED)
    assert np.abs(T_ref - Th)[p - 5:].max() > 0
    assert rel(T, T_ref) < 2e-4
