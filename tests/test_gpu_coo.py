"""The sparse exchange of cggm_solve (cggm_coo in and out, cggm_free_coo) through the C ABI.

The paper keeps Lambda and Theta in sparse form (Section 5); cggm_solve takes warm starts
as coordinate lists (Lambda as its upper triangle, Theta in full) and returns the solution
the same way, exact zeros dropped, in arrays the library allocates and cggm_free_coo
releases.  Checked here against the oracle's dense result on the 200 x 100 chain workload
(the method's bar), entry by entry against cggm_solve_dense (same kernels, so bit-equal),
and for the errors a coordinate list can carry.
"""
import ctypes

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


def check_list(coo, shape, upper):
    """Row-major order without repeats, inside the matrix, no stored zero."""
    r, c, v = coo
    assert r.dtype == np.int32 and c.dtype == np.int32 and v.dtype == np.float64
    assert np.all((r >= 0) & (r < shape[0]) & (c >= 0) & (c < shape[1]))
    if upper:
        assert np.all(r <= c)
    key = r.astype(np.int64) * shape[1] + c
    assert np.all(np.diff(key) > 0)
    assert np.all(v != 0) and np.all(np.isfinite(v))


def test_sparse_round_trip_matches_oracle(ctx):
    pr = synth.workload("chain-gauss-p200-q100-n100")
    p, q = pr.X.shape[1], pr.Y.shape[1]
    ref = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, max_iter=3000)
    # warm start: an interior iterate of the oracle, passed as coordinate lists
    mid = oracle.solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-12, max_iter=3)
    iu = np.nonzero(np.triu(mid.Lambda))
    wl = (iu[0], iu[1], mid.Lambda[iu])
    it = np.nonzero(mid.Theta)
    wt = (it[0], it[1], mid.Theta[it])
    o = cg.make_opts(precision=cg.CGGM_FP64, max_iter=3000)
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o, warm_Lambda=wl,
                       warm_Theta=wt)
    assert r.status == cg.CGGM_OK
    check_list(r.Lambda_coo, (q, q), True)
    check_list(r.Theta_coo, (p, q), False)
    # the lists hold exactly the nonzero entries of the dense solution they describe
    assert r.Lambda_coo[0].size == np.count_nonzero(np.triu(r.Lambda))
    assert r.Theta_coo[0].size == np.count_nonzero(r.Theta)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    f = oracle.objective(r.Lambda, r.Theta, Sxx, Sxy, Syy, pr.lam_L, pr.lam_T)
    assert (f - ref.f) / abs(ref.f) <= 1e-6
    assert rel(r.Lambda, ref.Lambda) <= 1e-4 and rel(r.Theta, ref.Theta) <= 1e-4
    # the same warm start given densely to cggm_solve_dense gives the same bits
    rd = ctx.cggm_solve_dense(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-7, opts=o,
                              warm_Lambda=mid.Lambda, warm_Theta=mid.Theta)
    np.testing.assert_array_equal(r.Lambda, rd.Lambda)
    np.testing.assert_array_equal(r.Theta, rd.Theta)
    # started from its own answer the solve stops at its first check
    r2 = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-6, opts=o,
                        warm_Lambda=r.Lambda_coo, warm_Theta=r.Theta_coo)
    assert r2.info["iterations"] <= 1


def test_repeated_entries_add_up_and_cold_start_equivalence(ctx):
    pr = synth.make_problem(30, 20, 40, seed=3, theta_nnz=3, lam=0.1)
    q = pr.Y.shape[1]
    o = cg.make_opts(precision=cg.CGGM_FP64, max_iter=50)
    cold = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-8, opts=o)
    # the identity listed as two halves of every diagonal entry, Theta as an empty list
    d = np.arange(q, dtype=np.int32)
    wl = (np.concatenate([d, d]), np.concatenate([d, d]), np.full(2 * q, 0.5))
    empty = (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    r = ctx.cggm_solve(pr.X, pr.Y, pr.lam_L, pr.lam_T, tol=1e-8, opts=o, warm_Lambda=wl,
                       warm_Theta=empty)
    np.testing.assert_array_equal(r.Lambda, cold.Lambda)
    np.testing.assert_array_equal(r.Theta, cold.Theta)


def test_bad_coordinate_lists(ctx):
    pr = synth.make_problem(12, 6, 20, seed=5, theta_nnz=2, lam=0.1)
    p, q = pr.X.shape[1], pr.Y.shape[1]
    eye = (np.arange(q), np.arange(q), np.ones(q))
    cases = [
        ((np.array([0, 3]), np.array([0, 1]), np.array([1.0, 0.1])), None, cg.CGGM_EINVAL),  # lower
        ((np.array([0]), np.array([q]), np.array([1.0])), None, cg.CGGM_EINVAL),              # col = q
        (eye, (np.array([p]), np.array([0]), np.array([1.0])), cg.CGGM_EINVAL),               # row = p
        (eye, (np.array([0]), np.array([-1]), np.array([1.0])), cg.CGGM_EINVAL),              # negative
        (eye, (np.array([1]), np.array([2]), np.array([np.nan])), cg.CGGM_ENONFINITE),
        ((np.arange(q), np.arange(q), -np.ones(q)), None, cg.CGGM_ENOTPD),
    ]
    for wl, wt, want in cases:
        with pytest.raises(cg.CGGMError) as e:
            ctx.cggm_solve(pr.X, pr.Y, 0.1, 0.1, warm_Lambda=wl, warm_Theta=wt)
        assert e.value.status == want
    # the context is still usable
    r = ctx.cggm_solve(pr.X, pr.Y, 0.1, 0.1, opts=cg.make_opts(precision=0, max_iter=5))
    assert np.all(np.isfinite(r.Lambda))


def test_outputs_are_empty_after_an_error_and_optional(ctx):
    """Through the raw C call: on an error the output lists are left empty; NULL outputs
    are allowed."""
    lib = cg.cggm._lib()
    pr = synth.make_problem(12, 6, 20, seed=5, theta_nnz=2, lam=0.1)
    n, p = pr.X.shape
    q = pr.Y.shape[1]
    X = np.ascontiguousarray(pr.X)
    Y = np.ascontiguousarray(pr.Y)
    outL, outT = cg.cggm_coo(), cg.cggm_coo()
    st = lib.cggm_solve(ctx._h, X.ctypes.data, cg.CGGM_F64, Y.ctypes.data, cg.CGGM_F64, n, p,
                        q, -1.0, 0.1, 0.0, None, None, None, ctypes.byref(outL),
                        ctypes.byref(outT), None)
    assert st == cg.CGGM_EINVAL
    assert outL.nnz == 0 and not outL.row and not outT.val
    st = lib.cggm_solve(ctx._h, X.ctypes.data, cg.CGGM_F64, Y.ctypes.data, cg.CGGM_F64, n, p,
                        q, 0.1, 0.1, 0.0, None, None, None, None, ctypes.byref(outT), None)
    assert st in (cg.CGGM_OK, cg.CGGM_EMAXITER)
    assert outT.nnz >= 0
    lib.cggm_free_coo(ctypes.byref(outT))
    assert outT.nnz == 0 and not outT.row
