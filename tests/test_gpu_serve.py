"""Regularisation-path server: a request's results are the same alone and in a mix of
concurrent requests, admission respects the memory budget, and the path's warm-started
solves reach what cold solves at the same lambda reach."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
cg = pytest.importorskip("paper_1509_04681_gb300")

GRID = [0.5, 0.3, 0.18, 0.1]


def prob(p, q, n, seed):
    pr = synth.make_problem(p, q, n, x_kind="gaussian", lam_kind="chain", theta_nnz=3, seed=seed)
    return pr.X, pr.Y


@pytest.fixture(scope="module")
def built():
    from paper_1509_04681_gb300 import build
    build.build()


def test_result_is_the_same_alone_and_in_the_mix(built):
    Xa, Ya = prob(60, 40, 50, seed=1)
    with cg.Server(0, slots=1) as s:
        ra = s.poll(s.submit(Xa, Ya, GRID, tol=1e-4, max_iter=300), wait=True)
    assert ra["status"] == 0
    others = [prob(120, 80, 90, seed=2), prob(40, 100, 60, seed=3), prob(200, 30, 70, seed=4)]
    with cg.Server(0, slots=4) as s:
        ids = [s.submit(X, Y, GRID, tol=1e-4, max_iter=300) for X, Y in others[:2]]
        ida = s.submit(Xa, Ya, GRID, tol=1e-4, max_iter=300)
        ids.append(s.submit(*others[2], GRID, tol=1e-4, max_iter=300))
        res = [s.poll(i, wait=True) for i in ids]
        rb = s.poll(ida, wait=True)
        st = s.stats()
    assert all(r["status"] == 0 for r in res) and rb["status"] == 0
    # the four requests overlapped on the device, and their coordinate passes shared launches
    spans = [(r["start_s"], r["finish_s"]) for r in res + [rb]]
    assert max(a for a, _ in spans) < min(b for _, b in spans)
    assert st["shared_launches"] > 0 and st["passes"] > st["pass_launches"], st
    # a pass's result does not depend on the SMs it shares a launch with: bit for bit
    np.testing.assert_array_equal(rb["Lambda"], ra["Lambda"])
    np.testing.assert_array_equal(rb["Theta"], ra["Theta"])


def test_admission_by_memory_budget(built):
    probs = [prob(100, 60, 80, seed=10 + k) for k in range(3)]
    fp = cg.footprint(80, 100, 60, cg.CGGM_MIXED)
    with cg.Server(0, slots=3, hbm_budget_bytes=int(fp * 1.5)) as s:  # room for one at a time
        ids = [s.submit(X, Y, GRID[:2], tol=1e-3, max_iter=100) for X, Y in probs]
        res = [s.poll(i, wait=True) for i in ids]
    assert all(r["status"] == 0 and r["footprint"] == fp for r in res)
    res.sort(key=lambda r: r["start_s"])
    for a, b in zip(res, res[1:]):
        assert b["start_s"] >= a["finish_s"] - 1e-6


def test_path_points_match_cold_solves(built):
    X, Y = prob(50, 30, 60, seed=20)
    with cg.Server(0, slots=2) as s:
        r = s.poll(s.submit(X, Y, GRID, tol=1e-7, max_iter=2000, precision=cg.CGGM_FP64), wait=True)
    with cg.Context(0) as ctx:
        for k, lam in enumerate(GRID):
            c = ctx.cggm_solve(X, Y, lam, lam, tol=1e-7,
                               opts=cg.make_opts(precision=cg.CGGM_FP64, max_iter=2000))
            f_path = ctx.cggm_objective(X, Y, r["Lambda"][k], r["Theta"][k], lam, lam)
            f_cold = ctx.cggm_objective(X, Y, c.Lambda, c.Theta, lam, lam)
            assert abs(f_path - f_cold) <= 1e-6 * abs(f_cold)
