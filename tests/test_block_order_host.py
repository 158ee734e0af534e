"""Visiting order and cache counts of Algorithm 2's blocked passes (cggm_block_order, host
code of the library; no GPU) against the oracle: the order is integer work, so it must
equal the oracle's bit for bit, and the counts must equal what the oracle's blocked passes
recorded while running (Sigma columns formed, misses)."""
import numpy as np
import pytest

import oracle
import paper_1509_04681_gb300 as cg
import synth
from oracle import blocks


@pytest.fixture(scope="module")
def state():
    pr = synth.make_problem(18, 14, 40, x_kind="gaussian", lam_kind="random3", theta_nnz=3,
                            lam=0.08, seed=5)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    r = oracle.solve(pr.X, pr.Y, 0.08, 0.08, tol=1e-12, max_iter=3)
    G_L, G_T, Sigma, Psi = oracle.gradients(r.Lambda, r.Theta, Sxx, Sxy, Syy)
    li, lj, ti, tj = oracle.active_sets(G_L, G_T, r.Lambda, r.Theta, 0.08, 0.08)
    return dict(X=pr.X, Sxy=Sxy, Syy=Syy, Lam=r.Lambda, Th=r.Theta,
                P=pr.X @ r.Theta @ Sigma, li=li, lj=lj, ti=ti, tj=tj)


def partitions(q):
    rng = np.random.default_rng(21)
    out = [np.zeros(q, dtype=np.int64), blocks.contiguous_partition(q, 4),
           np.arange(q)]                                   # one block, contiguous, singletons
    for k in (2, 3, 5):
        perm = rng.permutation(q)
        b = np.empty(q, dtype=np.int64)
        for z, part in enumerate(np.array_split(perm, k)):
            b[part] = z
        out.append(b)
    return out


def test_lambda_order_and_counts(state):
    q = state["Lam"].shape[0]
    for block in partitions(q):
        order, cols, miss = cg.block_order("lambda", q, state["li"], state["lj"], block)
        ref = blocks.lambda_block_order(state["li"], state["lj"], block)
        assert np.array_equal(order, ref)
        _, st = blocks.lambda_sweep_blocked(state["Lam"], state["P"], state["Syy"], state["li"],
                                            state["lj"], block, 0.08)
        assert (cols, miss) == (st.columns, st.misses)


def test_theta_order_and_counts(state):
    q = state["Lam"].shape[0]
    for block in partitions(q):
        order, cols, miss = cg.block_order("theta", q, state["ti"], state["tj"], block)
        ref = blocks.theta_block_order(state["ti"], state["tj"], block)
        assert np.array_equal(order, ref)
        _, st = blocks.theta_sweep_blocked(state["X"], state["Sxy"], state["Lam"], state["Th"],
                                           state["ti"], state["tj"], block, 0.08)
        assert (cols, miss) == (st.columns, st.misses)


def test_empty_list_and_errors():
    order, cols, miss = cg.block_order("lambda", 3, [], [], [0, 0, 1])
    assert order.size == 0 and (cols, miss) == (3, 0)
    with pytest.raises(cg.CGGMError):
        cg.block_order("lambda", 3, [2], [1], [0, 0, 1])         # i > j
    with pytest.raises(cg.CGGMError):
        cg.block_order("lambda", 3, [0], [1], [0, 2, 2])         # block 1 is empty
    with pytest.raises(cg.CGGMError):
        cg.block_order("theta", 3, [0], [3], [0, 0, 1])          # column out of range
    with pytest.raises(KeyError):
        cg.block_order("sigma", 3, [0], [1], [0, 0, 1])
