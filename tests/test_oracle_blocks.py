"""Pins of the oracle's block coordinate descent (Algorithm 2, Section 4) on the CPU.

The blocked passes hold only column blocks of Sigma, Psi and U (Lambda) or of Sigma and
V plus rows of S_xx formed from X (Theta).  Since each step is the exact minimiser of its
one-dimensional problem, a blocked pass must equal the sequential pass of Algorithm 1 over
the same coordinates taken in the blocked order; that sequential pass is pinned by
one-dimensional brute force (test_oracle_pins.py).  The cache rules are pinned by the
counts Section 4 states, and the whole blocked solve by the lambda = 0 closed form and by
Algorithm 1's optimum.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import blocks


def iterate(p=18, q=14, n=40, seed=5, iters=3, lam=0.08):
    """A point of Algorithm 1 a few iterations in (Lambda not diagonal, Theta nonzero)
    with its gradients, active sets and P = X Theta Sigma."""
    pr = synth.make_problem(p, q, n, x_kind="gaussian", lam_kind="random3", theta_nnz=3,
                            lam=lam, seed=seed)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    r = oracle.solve(pr.X, pr.Y, lam, lam, tol=1e-12, max_iter=iters)
    Lam, Th = r.Lambda, r.Theta
    G_L, G_T, Sigma, Psi = oracle.gradients(Lam, Th, Sxx, Sxy, Syy)
    li, lj, ti, tj = oracle.active_sets(G_L, G_T, Lam, Th, lam, lam)
    P = pr.X @ Th @ Sigma
    return dict(X=pr.X, Sxx=Sxx, Sxy=Sxy, Syy=Syy, Lam=Lam, Th=Th, Sigma=Sigma, Psi=Psi,
                li=li, lj=lj, ti=ti, tj=tj, P=P, lam=lam)


def random_partition(q, k, seed):
    """k non-empty blocks of scattered columns."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(q)
    block = np.empty(q, dtype=np.int64)
    for z, part in enumerate(np.array_split(perm, k)):
        block[part] = z
    return block


PARTITIONS = [("one block", 1, None), ("contiguous 4", None, 4), ("scattered 3", 3, 11),
              ("scattered 5", 5, 12), ("singletons", "q", 13)]


def make_partition(q, spec):
    _, k, arg = spec
    if k is None:
        return blocks.contiguous_partition(q, arg)
    if k == "q":
        return random_partition(q, q, arg)
    return random_partition(q, k, arg if arg is not None else 0)


@pytest.fixture(scope="module")
def it():
    return iterate()


@pytest.mark.parametrize("spec", PARTITIONS, ids=[s[0] for s in PARTITIONS])
def test_lambda_blocked_pass_equals_sequential_pass_in_block_order(it, spec):
    q = it["Lam"].shape[0]
    block = make_partition(q, spec)
    D, st = blocks.lambda_sweep_blocked(it["Lam"], it["P"], it["Syy"], it["li"], it["lj"],
                                        block, it["lam"])
    order = blocks.lambda_block_order(it["li"], it["lj"], block)
    D_seq = oracle.lambda_sweep(it["Sigma"], it["Psi"], it["Syy"], it["Lam"],
                                it["li"][order], it["lj"][order], it["lam"])
    assert np.count_nonzero(D_seq) > q        # the pass moves off-diagonal entries
    assert np.max(np.abs(D - D_seq)) <= 1e-11 * np.max(np.abs(D_seq))
    assert np.array_equal(D, D.T)


def test_lambda_one_block_is_algorithm_1_order(it):
    """With one block the blocked order is Algorithm 1's row-major order."""
    q = it["Lam"].shape[0]
    order = blocks.lambda_block_order(it["li"], it["lj"], np.zeros(q, dtype=np.int64))
    assert np.array_equal(order, np.arange(it["li"].size))


@pytest.mark.parametrize("spec", PARTITIONS, ids=[s[0] for s in PARTITIONS])
def test_theta_blocked_pass_equals_sequential_pass_in_block_order(it, spec):
    q = it["Lam"].shape[0]
    block = make_partition(q, spec)
    Th, st = blocks.theta_sweep_blocked(it["X"], it["Sxy"], it["Lam"], it["Th"], it["ti"],
                                        it["tj"], block, it["lam"])
    order = blocks.theta_block_order(it["ti"], it["tj"], block)
    Th_seq = oracle.theta_sweep(it["Sxx"], it["Sxy"], it["Sigma"], it["Th"],
                                it["ti"][order], it["tj"][order], it["lam"])
    assert np.any(Th_seq != it["Th"])
    assert np.max(np.abs(Th - Th_seq)) <= 1e-11 * np.max(np.abs(Th_seq))


def test_block_order_differs_from_row_major(it):
    """The pins above compare against the sequential pass in the blocked order; with more
    than one scattered block that order is not Algorithm 1's, and the passes differ."""
    q = it["Lam"].shape[0]
    block = random_partition(q, 3, 11)
    order = blocks.lambda_block_order(it["li"], it["lj"], block)
    assert not np.array_equal(order, np.arange(order.size))
    D_rm = oracle.lambda_sweep(it["Sigma"], it["Psi"], it["Syy"], it["Lam"], it["li"],
                               it["lj"], it["lam"])
    D_bl, _ = blocks.lambda_sweep_blocked(it["Lam"], it["P"], it["Syy"], it["li"], it["lj"],
                                          block, it["lam"])
    assert np.max(np.abs(D_rm - D_bl)) > 1e-8


def test_lambda_cache_rules(it):
    """Section 4.1: with every active coordinate inside a diagonal block, Sigma and Psi
    are formed once (q columns, no miss); each off-diagonal block pair with an active
    coordinate costs one miss and the columns of its second block."""
    q = it["Lam"].shape[0]
    block = blocks.contiguous_partition(q, 5)            # blocks of 5, 5, 4
    li, lj = np.triu_indices(q)
    inside = block[li] == block[lj]
    D, st = blocks.lambda_sweep_blocked(it["Lam"], it["P"], it["Syy"], li[inside], lj[inside],
                                        block, it["lam"])
    assert (st.columns, st.misses) == (q, 0)
    # add one coordinate in (C_0, C_2) and one in (C_1, C_2)
    extra_i = np.array([0, 6], dtype=np.int64)
    extra_j = np.array([12, 11], dtype=np.int64)
    li2 = np.concatenate([li[inside], extra_i])
    lj2 = np.concatenate([lj[inside], extra_j])
    D, st = blocks.lambda_sweep_blocked(it["Lam"], it["P"], it["Syy"], li2, lj2, block, it["lam"])
    assert st.misses == 2
    assert st.columns == q + 2 * 4


def test_theta_cache_rules(it):
    """Section 4.2: Sigma is formed once over the pass (q columns), and (S_xx)_i once per
    non-empty block (i, C_r) -- the count the partition is chosen to minimise."""
    q = it["Lam"].shape[0]
    for spec in PARTITIONS:
        block = make_partition(q, spec)
        _, st = blocks.theta_sweep_blocked(it["X"], it["Sxy"], it["Lam"], it["Th"], it["ti"],
                                           it["tj"], block, it["lam"])
        nonempty = len(set(zip(it["ti"].tolist(), block[it["tj"]].tolist())))
        assert st.columns == q
        assert st.misses == nonempty


def test_blocked_solve_lambda_zero_closed_form():
    """lambda = 0, n >= p + q: Algorithm 2 reaches the stationary point of Eq. 1,
    Lambda = (S_yy - S_xy^T S_xx^-1 S_xy)^-1, Theta = -S_xx^-1 S_xy Lambda."""
    pr = synth.make_problem(6, 4, 60, x_kind="gaussian", lam_kind="chain", theta_nnz=2,
                            lam=0.1, seed=3)
    Sxx, Sxy, Syy = oracle.covariances(pr.X, pr.Y)
    Lam_cf = np.linalg.inv(Syy - Sxy.T @ np.linalg.solve(Sxx, Sxy))
    Th_cf = -np.linalg.solve(Sxx, Sxy) @ Lam_cf
    part = lambda kind, q, i, j, mb: np.array([1, 0, 1, 0])      # scattered blocks
    r = blocks.solve_blocked(pr.X, pr.Y, 0.0, 0.0, max_block=2, tol=1e-12, max_iter=20000,
                             partition=part)
    assert r.converged
    assert np.max(np.abs(r.Lambda - Lam_cf)) < 1e-7 * np.max(np.abs(Lam_cf))
    assert np.max(np.abs(r.Theta - Th_cf)) < 1e-7 * np.max(np.abs(Th_cf))


def test_blocked_solve_reaches_algorithm_1_optimum():
    """With l1 penalties both algorithms minimise the same convex Eq. 1: the blocked solve
    ends at Algorithm 1's objective and support."""
    pr = synth.make_problem(12, 9, 40, x_kind="gaussian", lam_kind="chain", theta_nnz=2,
                            lam=0.1, seed=8)
    ref = oracle.solve(pr.X, pr.Y, 0.1, 0.1, tol=1e-10, max_iter=3000)
    r = blocks.solve_blocked(pr.X, pr.Y, 0.1, 0.1, max_block=4, tol=1e-10, max_iter=3000)
    assert r.converged and ref.converged
    assert abs(r.f - ref.f) <= 1e-10 * abs(ref.f)
    assert np.array_equal(np.abs(r.Lambda) > 1e-6, np.abs(ref.Lambda) > 1e-6)
    assert np.array_equal(np.abs(r.Theta) > 1e-6, np.abs(ref.Theta) > 1e-6)
    assert np.max(np.abs(r.Lambda - ref.Lambda)) <= 1e-5 * np.max(np.abs(ref.Lambda))
    # the objective decreases monotonically, as for Algorithm 1
    fs = [h.f for h in r.history]
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(fs, fs[1:]))


def test_partition_ids_are_checked():
    with pytest.raises(ValueError):
        blocks.block_lists(np.array([0, 2, 2]))
