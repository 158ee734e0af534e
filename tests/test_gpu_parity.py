"""CUDA path against the CPU oracle, step by step and for whole solves (needs a GPU).

Every test calls the library through the C ABI (ctypes binding) on inputs from the
seeded generators and compares element by element with the oracle on the same inputs.
Tolerances: double-precision kernels agree with the oracle to rounding (1e-9 relative
on the step outputs, the sums being reordered); single-precision caches (mixed) to
1e-4 relative on the steps.  Whole solves are compared by the acceptance bar of the
method: relative objective gap <= 1e-6, max |dLambda|, |dTheta| <= 1e-4 max|entry|, same
support above 1e-3.
"""
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


def problem(p, q, n, seed, **kw):
    kw.setdefault("theta_nnz", 3)
    return synth.make_problem(p, q, n, seed=seed, **kw)


def state_at(pr, iters=2):
    """An interior iterate of the oracle (nonzero Theta, non-identity Lambda)."""
    r = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, max_iter=iters)
    return r.Lambda, r.Theta


# ------------------------------------------------------------------------------------
# Cholesky, log det, Sigma
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("q", [1, 63, 64, 65, 200, 333])
def test_cholesky_logdet_sigma(ctx, q):
    rng = np.random.default_rng(q)
    A = rng.standard_normal((q, q + 5))
    Lam = A @ A.T / q + 0.5 * np.eye(q)
    L, ld, S = ctx.cggm_cholesky(Lam)
    L_ref = np.linalg.cholesky(Lam)
    assert rel(L, L_ref) < 1e-12
    assert abs(ld - 2 * np.log(np.diag(L_ref)).sum()) < 1e-11 * max(1, abs(ld))
    assert rel(S, np.linalg.inv(Lam)) < 1e-10


def test_cholesky_not_pd_is_reported(ctx):
    Lam = np.diag([1.0, 2.0, -1.0, 3.0])
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_cholesky(Lam)
    assert e.value.status == cg.CGGM_ENOTPD


# ------------------------------------------------------------------------------------
# gradients and objective
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(30, 20, 25), (130, 70, 90), (7, 1, 12), (1, 5, 9)])
def test_grad_and_objective(ctx, shape):
    p, q, n = shape
    pr = problem(p, q, n, seed=p + q)
    Lam, Th = state_at(pr)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    G_L, G_T, _, _ = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    gL, gT = ctx.cggm_grad(pr.X, pr.Y, Lam, Th)
    assert rel(gL, G_L) < 1e-10
    assert rel(gT, G_T) < 1e-10
    for pen in (True, False):
        f_ref = oracle.objective(Lam, Th, Sxx, Sxy, Syy, 0.1, 0.2, pen)
        f = ctx.cggm_objective(pr.X, pr.Y, Lam, Th, 0.1, 0.2, pen)
        assert abs(f - f_ref) < 1e-11 * abs(f_ref)


def test_grad_and_objective_sparse_theta_edges(ctx):
    """R = X Theta is formed over Theta's nonzeros (scanned in chunks of 256 rows, summed
    over n in passes of 1024): p = 300 and n = 1300 take two of each with a ragged tail;
    Theta has an empty column, a dense one, one whose only entry is in the last row, and
    scattered entries elsewhere; and Theta = 0."""
    p, q, n = 300, 9, 1300
    pr = problem(p, q, n, seed=77)
    rng = np.random.default_rng(77)
    Th = np.where(rng.random((p, q)) < 0.05, rng.standard_normal((p, q)) * 0.1, 0.0)
    Th[:, 0] = 0.0
    Th[:, 1] = rng.standard_normal(p) * 0.05
    Th[:, 2] = 0.0
    Th[p - 1, 2] = 0.3
    Lam = synth.chain_precision(q).toarray()
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    for T in (Th, np.zeros((p, q))):
        G_L, G_T, _, _ = oracle.gradients(Lam, T, Sxx, Sxy, Syy)
        gL, gT = ctx.cggm_grad(pr.X, pr.Y, Lam, T)
        assert rel(gL, G_L) < 1e-10
        assert rel(gT, G_T) < 1e-10
        f_ref = oracle.objective(Lam, T, Sxx, Sxy, Syy, 0.1, 0.2)
        f = ctx.cggm_objective(pr.X, pr.Y, Lam, T, 0.1, 0.2)
        assert abs(f - f_ref) < 1e-11 * abs(f_ref)


# ------------------------------------------------------------------------------------
# active sets: integer work, bit-exact
# ------------------------------------------------------------------------------------
@pytest.mark.parametrize("pen", [True, False])
def test_active_sets_bit_exact(ctx, pen):
    pr = problem(90, 70, 60, seed=5)
    Lam, Th = state_at(pr)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    G_L, G_T, _, _ = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    ref = oracle.active_sets(G_L, G_T, Lam, Th, 0.1, 0.1, pen)
    got = ctx.cggm_active_sets(G_L, G_T, Lam, Th, 0.1, 0.1, pen)
    for a, b in zip(got, ref):
        np.testing.assert_array_equal(a, b)


def test_active_sets_empty_and_full(ctx):
    q, p = 5, 4
    G_L = np.zeros((q, q)); G_T = np.zeros((p, q))
    li, lj, ti, tj = ctx.cggm_active_sets(G_L, G_T, np.eye(q), np.zeros((p, q)), 1.0, 1.0)
    assert list(zip(li, lj)) == [(i, i) for i in range(q)] and len(ti) == 0
    li, lj, ti, tj = ctx.cggm_active_sets(G_L + 5, G_T + 5, np.eye(q), np.zeros((p, q)), 1.0, 1.0)
    assert len(li) == q * (q + 1) // 2 and len(ti) == p * q


# ------------------------------------------------------------------------------------
# coordinate passes
# ------------------------------------------------------------------------------------
def lambda_inputs(p, q, n, seed, lam=0.05):
    pr = problem(p, q, n, seed=seed)
    Lam, Th = state_at(pr)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    G_L, G_T, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    li, lj, ti, tj = oracle.active_sets(G_L, G_T, Lam, Th, lam, lam)
    return pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi, li, lj, ti, tj


@pytest.mark.parametrize("shape", [(40, 37, 30), (120, 150, 80), (60, 1, 40)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
def test_lambda_sweep(ctx, shape, prec, tol):
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi, li, lj, _, _ = lambda_inputs(*shape, seed=11)
    assert len(li) > 128 or shape[1] == 1  # several batches and a ragged tail
    D_ref = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.05)
    D = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.05, precision=prec)
    assert rel(D, D_ref) < tol
    np.testing.assert_array_equal(D, D.T)


def test_lambda_sweep_sparse_random_order(ctx):
    """Scattered active coordinates (not whole rows), and the unpenalised diagonal."""
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi, _, _, _, _ = lambda_inputs(50, 90, 60, seed=3)
    rng = np.random.default_rng(0)
    iu, ju = np.triu_indices(90)
    keep = rng.uniform(size=iu.size) < 0.15
    keep[iu == ju] = True
    li, lj = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    for pen in (True, False):
        D_ref = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.03, pen)
        D = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.03, pen, precision=0)
        assert rel(D, D_ref) < 1e-9


@pytest.mark.parametrize("shape", [(40, 37, 30), (150, 120, 80), (1, 30, 20), (70, 1, 50)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
def test_theta_sweep(ctx, shape, prec, tol):
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi, _, _, ti, tj = lambda_inputs(*shape, seed=17)
    T_ref = oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti, tj, 0.05)
    T = ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, ti, tj, 0.05, precision=prec)
    assert rel(T, T_ref) < tol


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-4)])
@pytest.mark.parametrize("length", [1032, 1030])
def test_sweeps_long_rows(ctx, prec, tol, length):
    """Rows longer than one shared-memory chunk of the dot-product ring (1032 entries: several
    chunks in float and in double), and a row length that is not a whole number of 16-byte
    words (1030: direct loads instead of bulk copies)."""
    def inputs(p, q, seed):
        # the true parameters, scaled, stand in for an interior iterate (an oracle solve at
        # these sizes would take longer than the check itself)
        pr = problem(p, q, 40, seed=seed)
        Lam = pr.Lambda_true.toarray()
        Th = 0.5 * pr.Theta_true.toarray()
        Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
        G_L, G_T, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
        return pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi

    q = length
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi = inputs(24, q, 5)
    iu, ju = np.triu_indices(q)
    keep = (iu < 2) | ((iu == ju) & (iu % 97 == 0)) | ((iu == q - 3) & (ju > q - 40))
    li, lj = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    D_ref = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.05)
    D = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li, lj, 0.05, precision=prec)
    assert np.abs(D_ref).max() > 0
    assert rel(D, D_ref) < tol
    p = length
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi = inputs(p, 24, 6)
    rows = np.array([0, 3, p - 7, p - 1])
    ti = np.repeat(rows, 24).astype(np.int32)
    tj = np.tile(np.arange(24), rows.size).astype(np.int32)
    T_ref = oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti, tj, 0.02)
    T = ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, ti, tj, 0.02, precision=prec)
    assert np.abs(T_ref - Th).max() > 0
    assert rel(T, T_ref) < tol


def test_sweeps_with_empty_active_set(ctx):
    pr, Lam, Th, Sxx, Sxy, Syy, Sigma, Psi, _, _, _, _ = lambda_inputs(20, 10, 15, seed=2)
    e = np.zeros(0, dtype=np.int32)
    assert np.all(ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, e, e, 0.1) == 0)
    np.testing.assert_array_equal(ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, e, e, 0.1), Th)


# ------------------------------------------------------------------------------------
# whole solves
# ------------------------------------------------------------------------------------
def check_solution(pr, r_gpu, ref, f_star):
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    f_gpu = oracle.objective(r_gpu.Lambda, r_gpu.Theta, Sxx, Sxy, Syy, pr.lam_L, pr.lam_T)
    gap = (f_gpu - f_star) / abs(f_star)
    assert gap <= 1e-6, gap
    assert rel(r_gpu.Lambda, ref.Lambda) <= 1e-4
    assert rel(r_gpu.Theta, ref.Theta) <= 1e-4
    for A, B in ((r_gpu.Lambda, ref.Lambda), (r_gpu.Theta, ref.Theta)):
        sa, sb = np.abs(A) > 1e-3, np.abs(B) > 1e-3
        # entries within rounding of the 1e-3 cut may fall either side
        border = np.abs(np.abs(B) - 1e-3) < 1e-5
        assert np.all((sa == sb) | border)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_small_chain_matches_oracle(ctx, prec):
    pr = synth.workload("chain-gauss-p200-q100-n100")
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    f_star = ref.f
    o = cg.make_opts(precision=prec, max_iter=3000)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o)
    check_solution(pr, r, ref, f_star)


def test_solve_batch_of_512_matches_oracle(ctx):
    """The mixed path with batches of 512 coordinates (coefficient panels streamed through two
    shared-memory buffers in phase B) on the 200 x 100 workload, by the same bar."""
    pr = synth.workload("chain-gauss-p200-q100-n100")
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    o = cg.make_opts(precision=cg.CGGM_MIXED, max_iter=3000, sweep_batch=512)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o)
    check_solution(pr, r, ref, ref.f)


def test_solve_with_tuned_batch_size(ctx):
    """sweep_batch = auto: the first iteration of a new size class times the Lambda pass at
    every candidate batch size and keeps the fastest; the solve meets the same bar."""
    pr = synth.workload("chain-gauss-p200-q100-n100")
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    o = cg.make_opts(precision=cg.CGGM_MIXED, max_iter=3000, sweep_batch=cg.CGGM_SWEEP_BATCH_AUTO)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o)
    check_solution(pr, r, ref, ref.f)
    assert r.info["m_lambda"] > 0
    tuned = [cg.tuned_batch(100, m, cg.CGGM_MIXED) for m in (r.info["m_lambda"], 5050)]
    assert any(b in (64, 128, 256, 512) for b in tuned)
    assert cg.tuned_batch(100, 10 ** 9, cg.CGGM_MIXED) == 0  # a class never seen
    assert cg.tuned_batch(0, 10, cg.CGGM_MIXED) == -1


def test_solve_first_iterates_track_oracle(ctx):
    """FP64 path: the objective after each of the first iterations equals the oracle's."""
    pr = problem(60, 40, 50, seed=8, lam=0.1)
    for k in (1, 2, 5):
        ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, max_iter=k)
        r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12,
                           opts=cg.make_opts(precision=0, max_iter=k))
        assert rel(r.Lambda, ref.Lambda) < 1e-8
        assert rel(r.Theta, ref.Theta) < 1e-8


def test_solve_warm_start_and_unpenalised_diagonal(ctx):
    pr = problem(30, 20, 40, seed=4, lam=0.2)
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-8, max_iter=2000,
                       penalize_diag=False)
    o = cg.make_opts(precision=0, penalize_diag=0, max_iter=2000)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-8, opts=o)
    assert rel(r.Lambda, ref.Lambda) < 1e-5
    # warm start from the answer converges immediately
    r2 = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-6, opts=o,
                        warm_Lambda=r.Lambda, warm_Theta=r.Theta)
    assert r2.info["iterations"] <= 2


def test_solve_degenerate_cases(ctx):
    # huge penalties: Theta stays 0, Lambda diagonal
    pr = problem(10, 6, 20, seed=9)
    r = ctx.cggm_solve(pr.X, pr.Y, 100.0, 100.0, tol=1e-8,
                       opts=cg.make_opts(precision=0, max_iter=500))
    assert np.all(r.Theta == 0)
    assert np.all(r.Lambda[~np.eye(6, dtype=bool)] == 0)
    # p = q = 1
    x = np.random.default_rng(0).standard_normal((50, 1))
    y = -0.7 * x + 0.3 * np.random.default_rng(1).standard_normal((50, 1))
    r = ctx.cggm_solve(x, y, 0.05, 0.1, tol=1e-10, opts=cg.make_opts(precision=0))
    ref = oracle.solve(x, y, 0.05, 0.1, tol=1e-10, max_iter=1000)
    assert abs(r.Lambda[0, 0] - ref.Lambda[0, 0]) < 1e-7 * ref.Lambda[0, 0]


def test_solve_rejects_bad_input(ctx):
    pr = problem(10, 6, 20, seed=9)
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_solve(pr.X, pr.Y, -1.0, 0.1)
    assert e.value.status == cg.CGGM_EINVAL
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_solve(pr.X, pr.Y, 0.1, 0.1, warm_Lambda=-np.eye(6))
    assert e.value.status == cg.CGGM_ENOTPD
    X = pr.X.copy(); X[3, 4] = np.nan
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_solve(X, pr.Y, 0.1, 0.1)
    assert e.value.status == -8


def test_solve_line_search_exhaustion(ctx):
    """Forced line-search exhaustion (pinned on the oracle: with sigma = 1 a full step never
    meets the Armijo rule, the objective being strictly convex along the direction): one
    trial gives CGGM_ELINESEARCH, and the context stays usable."""
    pr = problem(6, 5, 40, seed=13)
    o = cg.make_opts(precision=cg.CGGM_FP64, ls_sigma=1.0, ls_max_trials=1, max_iter=3)
    with pytest.raises(cg.CGGMError) as e:
        ctx.cggm_solve(pr.X, pr.Y, 0.1, 0.1, tol=1e-8, opts=o)
    assert e.value.status == cg.CGGM_ELINESEARCH
    r = ctx.cggm_solve(pr.X, pr.Y, 0.1, 0.1, tol=1e-8,
                       opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=3))
    assert np.all(np.isfinite(r.Lambda)) and r.info["iterations"] >= 1


def test_device_inputs(ctx):
    torch = pytest.importorskip("torch")
    pr = problem(30, 20, 40, seed=12)
    Xd = torch.tensor(pr.X, device="cuda:0", dtype=torch.float32)
    Yd = torch.tensor(pr.Y, device="cuda:0", dtype=torch.float32)
    r1 = ctx.cggm_solve(Xd, Yd, pr.lam_L, pr.lam_T, tol=1e-6, opts=cg.make_opts(precision=0))
    r2 = ctx.cggm_solve(pr.X.astype(np.float32), pr.Y.astype(np.float32), pr.lam_L, pr.lam_T,
                        tol=1e-6, opts=cg.make_opts(precision=0))
    np.testing.assert_array_equal(r1.Lambda, r2.Lambda)


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_with_sxx_in_row_chunks_matches_oracle(ctx, prec):
    """S_xx held 37 rows at a time (200 inputs: five full chunks and a ragged sixth, each
    formed from X before the Theta pass continues over its rows): the whole solve meets the
    method's bar against the oracle, and in double precision stays within rounding of the
    solve that holds S_xx whole."""
    pr = synth.workload("chain-gauss-p200-q100-n100")
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    o = cg.make_opts(precision=prec, max_iter=3000, sxx_rows=37)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o)
    check_solution(pr, r, ref, ref.f)
    if prec == 0:
        for k in (1, 3):
            a = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12,
                               opts=cg.make_opts(precision=0, max_iter=k, sxx_rows=37))
            b = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, max_iter=k)
            assert rel(a.Theta, b.Theta) < 1e-8 and rel(a.Lambda, b.Lambda) < 1e-8


def test_theta_pass_out_of_row_order(ctx):
    """The step-level Theta pass with a list that is not row-major (distinct coordinates,
    rows jumping back and forth) equals the oracle's pass in that order.  (Its rows fit one
    S_xx chunk here; lists over several chunks are covered at p = 40000 in
    test_gpu_maxsize.py.)"""
    pr = problem(50, 12, 30, seed=21)
    Lam, Th = state_at(pr)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    Sigma = np.linalg.inv(Lam)
    rng = np.random.default_rng(21)
    flat = rng.permutation(50 * 12)[:300]
    ti = (flat // 12).astype(np.int32)
    tj = (flat % 12).astype(np.int32)
    want = oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti, tj, 0.05)
    got = ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, ti, tj, 0.05, precision=cg.CGGM_FP64)
    assert rel(got, want) < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_clustered_network_family_matches_oracle(ctx, prec):
    """The paper's random graphs with clustering (Section 5: clusters of 250, average degree
    10, Theta on 100 sqrt(p) inputs with 10 q edges, n = 200) through cggm_solve, by the
    method's bar against the oracle."""
    pr = synth.clustered_problem(300, 250, n=200, lam=0.15, seed=2)
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7,
                       opts=cg.make_opts(precision=prec, max_iter=3000))
    check_solution(pr, r, ref, ref.f)
