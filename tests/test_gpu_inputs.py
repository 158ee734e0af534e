"""Input element types of X and Y (Section 2.1): int8 genotype counts standardised on the
device, bfloat16 and float32 inputs, each against the same matrix given in float64 (needs
a GPU).  The standardisation reference is its definition written out here: per column,
(x - mean) / population sd."""
import numpy as np
import pytest

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


def standardise(raw):
    x = raw.astype(np.float64)
    sd = x.std(axis=0)
    return np.where(sd > 0, (x - x.mean(axis=0)) / np.where(sd > 0, sd, 1.0), 0.0)


def genotype_problem(p=70, q=30, n=90, seed=3):
    pr = synth.make_problem(p, q, n, x_kind="genotype", seed=seed, theta_nnz=3)
    Lam = pr.Lambda_true.toarray()
    Th = 0.5 * pr.Theta_true.toarray()
    return pr, Lam, Th


def test_int8_genotypes_standardised_on_device(ctx):
    pr, Lam, Th = genotype_problem()
    raw = pr.X_raw
    assert raw.dtype == np.int8 and set(np.unique(raw)) <= {0, 1, 2}
    Xs = standardise(raw)
    np.testing.assert_allclose(Xs, pr.X, rtol=0, atol=1e-12)  # the generator agrees
    gL8, gT8 = ctx.cggm_grad(raw, pr.Y, Lam, Th)
    gL, gT = ctx.cggm_grad(Xs, pr.Y, Lam, Th)
    assert rel(gL8, gL) < 1e-12 and rel(gT8, gT) < 1e-12
    f8 = ctx.cggm_objective(raw, pr.Y, Lam, Th, pr.lam_L, pr.lam_T)
    f = ctx.cggm_objective(Xs, pr.Y, Lam, Th, pr.lam_L, pr.lam_T)
    assert abs(f8 - f) <= 1e-12 * abs(f)
    for prec in (cg.CGGM_FP64, cg.CGGM_MIXED):
        o = cg.make_opts(precision=prec, max_iter=4)
        r8 = ctx.cggm_solve(raw, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, opts=o)
        r = ctx.cggm_solve(Xs, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, opts=o)
        assert abs(r8.info["f"] - r.info["f"]) <= 1e-9 * abs(r.info["f"])
        assert rel(r8.Lambda, r.Lambda) < 1e-6 and rel(r8.Theta, r.Theta) < 1e-6


def test_constant_genotype_column_becomes_zero(ctx):
    pr, Lam, Th = genotype_problem(seed=4)
    raw = pr.X_raw.copy()
    raw[:, 5] = 1
    Th[5, :] = 0.0
    Xs = standardise(raw)
    assert np.all(Xs[:, 5] == 0.0)
    gL8, gT8 = ctx.cggm_grad(raw, pr.Y, Lam, Th)
    gL, gT = ctx.cggm_grad(Xs, pr.Y, Lam, Th)
    assert rel(gL8, gL) < 1e-12 and rel(gT8, gT) < 1e-12
    assert np.all(gT8[5] == 0.0)
    r = ctx.cggm_solve(raw, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12,
                       opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=3))
    assert np.all(r.Theta[5] == 0.0)


def test_bf16_and_f32_inputs_equal_their_f64_values(ctx):
    torch = pytest.importorskip("torch")
    pr, Lam, Th = genotype_problem(seed=5)
    Xb = torch.from_numpy(pr.X).to(torch.bfloat16)
    Yb = torch.from_numpy(pr.Y).to(torch.bfloat16)
    Xv, Yv = Xb.double().numpy(), Yb.double().numpy()  # the values bf16 holds, exactly
    gLb, gTb = ctx.cggm_grad(Xb, Yb, Lam, Th)
    gL, gT = ctx.cggm_grad(Xv, Yv, Lam, Th)
    np.testing.assert_array_equal(gLb, gL)
    np.testing.assert_array_equal(gTb, gT)
    X32, Y32 = pr.X.astype(np.float32), pr.Y.astype(np.float32)
    gL32, gT32 = ctx.cggm_grad(X32, Y32, Lam, Th)
    gL, gT = ctx.cggm_grad(X32.astype(np.float64), Y32.astype(np.float64), Lam, Th)
    np.testing.assert_array_equal(gL32, gL)
    np.testing.assert_array_equal(gT32, gT)


def test_genotype_y_is_rejected(ctx):
    pr, Lam, Th = genotype_problem(seed=6)
    with pytest.raises(cg.CGGMError):
        ctx.cggm_grad(pr.X, pr.X_raw[:, :30].copy(), Lam, Th)
