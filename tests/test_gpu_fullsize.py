"""The 5000 x 5000 genotype workload at full size (needs a GPU).

The benchmark times this workload in the mixed-precision path with batches of 256.  The
whole pass there is too long for the oracle, so this test checks what the oracle can do at
this size: the gradients (Eq. 3) and the objective (Eq. 1) in full against the oracle's
double-precision formulas, and each coordinate pass, in the benchmark's launch configuration
(float caches, B = 256, one CTA per SM), over bounded prefixes of the real active sets
against the oracle's sequential pass on the same prefixes.  Inputs are generated (the true
Lambda and half the true Theta as the current point); none come from the CUDA path."""
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


@pytest.fixture(scope="module")
def big():
    pr = synth.workload("chain-geno-p5000-q5000-n1000")
    Lam = pr.Lambda_true.toarray()
    Th = 0.5 * pr.Theta_true.toarray()
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    G_L, G_T, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    return pr, Lam, Th, Sxx, Sxy, Syy, G_L, G_T, Sigma, Psi


def rel(a, b):
    return np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b)))


def test_gradients_and_objective_full_size(ctx, big):
    pr, Lam, Th, Sxx, Sxy, Syy, G_L, G_T, Sigma, Psi = big
    gL, gT = ctx.cggm_grad(pr.X_raw, pr.Y, Lam, Th)  # int8 genotypes, standardised on device
    assert rel(gL, G_L) < 1e-9 and rel(gT, G_T) < 1e-9
    f = ctx.cggm_objective(pr.X_raw, pr.Y, Lam, Th, pr.lam_L, pr.lam_T)
    f_ref = oracle.objective(Lam, Th, Sxx, Sxy, Syy, pr.lam_L, pr.lam_T)
    assert abs(f - f_ref) <= 1e-10 * abs(f_ref)


def test_lambda_pass_prefix_full_size(ctx, big):
    pr, Lam, Th, Sxx, Sxy, Syy, G_L, G_T, Sigma, Psi = big
    li, lj, _, _ = oracle.active_sets(G_L, G_T, Lam, Th, pr.lam_L, pr.lam_T)
    assert len(li) > 100000  # the real active set is large; a prefix of it is checked
    k = 4000  # ~16 batches of 256 with a ragged tail, rows of 5000 entries
    D_ref = oracle.lambda_sweep(Sigma, Psi, Syy, Lam, li[:k], lj[:k], pr.lam_L)
    D = ctx.cggm_lambda_sweep(Sigma, Psi, Syy, Lam, li[:k], lj[:k], pr.lam_L,
                              precision=cg.CGGM_MIXED)
    assert np.abs(D_ref).max() > 0
    assert rel(D, D_ref) < 2e-4


def test_theta_pass_prefix_full_size(ctx, big):
    pr, Lam, Th, Sxx, Sxy, Syy, G_L, G_T, Sigma, Psi = big
    _, _, ti, tj = oracle.active_sets(G_L, G_T, Lam, Th, pr.lam_L, pr.lam_T)
    # an early stretch and a late one (the late rows' dot products run over ~p entries)
    late = np.flatnonzero(ti >= 4990)[:1500]
    sel = np.concatenate([np.arange(1500), late])
    T_ref = oracle.theta_sweep(Sxx, Sxy, Sigma, Th, ti[sel], tj[sel], pr.lam_T)
    T = ctx.cggm_theta_sweep(pr.X, Sxy, Sigma, Th, ti[sel], tj[sel], pr.lam_T,
                             precision=cg.CGGM_MIXED)
    assert np.abs(T_ref - Th).max() > 0
    assert rel(T, T_ref) < 2e-4
