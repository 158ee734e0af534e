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


def test_block_regime_host_plan_end_to_end():
    """The host pieces of the block regime in sequence on a random network of average degree
    4 with 3000 outputs (the shape of the large workloads' Lambda): partition its graph,
    order the active coordinates by block pairs, permute Lambda so every block is
    contiguous, analyse the sparse factor and lay out its supernodes.  Each output is a
    valid input of the next and the pieces agree on their sizes."""
    import scipy.sparse as sp
    q = 3000
    Lam = synth.random_sparse_precision(q, 4.0, np.random.default_rng(30)).tocsr()
    U = sp.triu(Lam).tocoo()
    li, lj = U.row.astype(np.int32), U.col.astype(np.int32)
    off = li != lj
    block, k, cut = cg.partition_columns(q, li[off], lj[off], 256)
    assert k >= -(-q // 256)
    order, cols, miss = cg.block_order("lambda", q, li, lj, block)
    assert np.array_equal(np.sort(order), np.arange(li.size)) and cols >= q
    perm = np.argsort(block, kind="stable").astype(np.int32)
    rp, ci, v = cg.permute_csr(q, Lam.indptr, Lam.indices, Lam.data, perm)
    P = sp.csr_matrix((v, ci, rp), shape=(q, q))
    assert np.array_equal(P.toarray(), Lam.toarray()[np.ix_(perm, perm)])
    sizes = np.bincount(block)
    starts = np.r_[0, np.cumsum(sizes)]
    assert np.array_equal(np.sort(block)[starts[:-1]], np.arange(k))   # blocks contiguous
    pv, parent, cc, nnz = cg.chol_symbolic(q, rp, ci, cg.CGGM_ORDER_AMD)
    ss = cg.chol_supernodes(parent, cc)
    rows_ptr, rows = cg.chol_structure(q, rp, ci, pv, parent, cc, ss)
    assert ss[0] == 0 and ss[-1] == q and rows_ptr[-1] == cc[ss[:-1]].sum()
    # every supernode's rows start with its own columns and stay inside the matrix
    for s in range(len(ss) - 1):
        r = rows[rows_ptr[s]:rows_ptr[s + 1]]
        assert np.array_equal(r[:ss[s + 1] - ss[s]], np.arange(ss[s], ss[s + 1]))
        assert r[-1] < q


def test_block_count_rule():
    """Section 4's rule: the least k whose block columns fit (Lambda holds 4 q ceil(q/k)
    values, Theta q ceil(q/k))."""
    q, b = 200000, 4
    budget = 3_300_000_000                        # a few GB for the blocks
    k, mb = cg.block_count("lambda", q, b, budget)
    assert 4 * q * -(-q // k) * b <= budget           # k blocks fit ...
    assert k == 1 or 4 * q * -(-q // (k - 1)) * b > budget   # ... and k - 1 would not
    assert mb == -(-q // k)
    k, mb = cg.block_count("theta", q, b, budget)
    assert q * -(-q // k) * b <= budget and (k == 1 or q * -(-q // (k - 1)) * b > budget)
    assert cg.block_count("lambda", 1000, 8, 10 ** 12) == (1, 1000)   # everything fits
    with pytest.raises(cg.CGGMError) as e:
        cg.block_count("lambda", 1000, 8, 4 * 1000 * 8 - 1)            # not one column
    assert e.value.status == cg.CGGM_ENOMEM
    with pytest.raises(cg.CGGMError):
        cg.block_count("lambda", 0, 8, 10 ** 9)
