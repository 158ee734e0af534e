"""Column partitions for the block coordinate descent of Algorithm 2 (Section 4), through
the C ABI (host code of the library; no GPU).

Several partitions can be equally good, so these tests check what is fixed: every column
in one block of at most max_block columns, ids 0..k-1 with no empty block, the reported
cut and row-block count against their definitions, determinism, and the optimum on
graphs where it has a closed form (a path, disjoint cliques, two-vertex weights).  On a
planted partition the cut must be no worse than the planted one, and on a grid no worse
than strips.
"""
import numpy as np
import pytest

import paper_1509_04681_gb300 as cg


def check_valid(block, k, q, max_block):
    assert block.shape == (q,)
    if q == 0:
        assert k == 0
        return
    assert block.min() == 0 and block.max() == k - 1
    sizes = np.bincount(block, minlength=k)
    assert np.all(sizes >= 1) and np.all(sizes <= max_block)
    # ids numbered by the lowest column they hold
    firsts = [int(np.flatnonzero(block == b)[0]) for b in range(k)]
    assert firsts == sorted(firsts)


def cut_of(block, ei, ej, w=None):
    w = np.ones(len(ei)) if w is None else np.asarray(w)
    ei, ej = np.asarray(ei), np.asarray(ej)
    off = ei != ej
    return float(np.sum(w[off] * (block[ei[off]] != block[ej[off]])))


def er_graph(q, m, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, q, m), rng.integers(0, q, m)


@pytest.mark.parametrize("q,m,cap", [(1, 0, 1), (7, 10, 1), (50, 200, 7), (300, 1500, 64),
                                     (300, 1500, 300), (301, 900, 1000), (2000, 6000, 128)])
def test_valid_and_cut_matches_definition(q, m, cap):
    ei, ej = er_graph(q, m, q + m + cap)
    block, k, cut = cg.partition_columns(q, ei, ej, cap)
    check_valid(block, k, q, cap)
    assert cut == pytest.approx(cut_of(block, ei, ej), abs=1e-9)
    if cap >= q:
        assert k == 1 and cut == 0.0


def test_empty_graph_and_no_columns():
    block, k, cut = cg.partition_columns(0, [], [], 4)
    assert block.size == 0 and k == 0 and cut == 0.0
    block, k, cut = cg.partition_columns(10, [], [], 4)     # ten isolated columns
    check_valid(block, k, 10, 4)
    assert k == 3 and cut == 0.0


def test_path_with_shuffled_labels_reaches_the_optimum():
    """A path on q vertices needs ceil(q / B) blocks of at most B, hence at least
    ceil(q / B) - 1 cut edges; the partitioner finds that optimum whatever the labels."""
    rng = np.random.default_rng(1)
    for q, cap in [(1000, 64), (999, 100), (130, 13), (64, 64), (65, 64)]:
        lab = rng.permutation(q)
        ei, ej = lab[:-1], lab[1:]
        block, k, cut = cg.partition_columns(q, ei, ej, cap)
        check_valid(block, k, q, cap)
        kmin = -(-q // cap)
        assert k == kmin
        assert cut == kmin - 1


def test_disjoint_cliques_stay_whole():
    """40 cliques of 8 scattered labels, blocks of 32: a cut of zero exists (four whole
    cliques per block) and is found."""
    rng = np.random.default_rng(2)
    q, c = 320, 8
    lab = rng.permutation(q).reshape(-1, c)
    ei, ej = [], []
    for g in lab:
        a, b = np.triu_indices(c, 1)
        ei += g[a].tolist()
        ej += g[b].tolist()
    block, k, cut = cg.partition_columns(q, ei, ej, 32)
    check_valid(block, k, q, 32)
    assert cut == 0.0 and k == 10
    for g in lab:
        assert len(set(block[g].tolist())) == 1


def test_weights_decide():
    """a - b of weight 10, b - c of weight 1, blocks of two: {a, b}, {c}, cut 1."""
    block, k, cut = cg.partition_columns(3, [0, 1], [1, 2], 2, w=[10.0, 1.0])
    assert block[0] == block[1] != block[2] and cut == 1.0
    block, k, cut = cg.partition_columns(3, [0, 1], [1, 2], 2, w=[1.0, 10.0])
    assert block[1] == block[2] != block[0] and cut == 1.0


def test_repeated_edges_and_self_loops():
    block, k, cut = cg.partition_columns(4, [0, 0, 1, 2, 3, 2], [1, 1, 1, 3, 3, 3], 2)
    check_valid(block, k, 4, 2)
    assert cut == 0.0 and block[0] == block[1] and block[2] == block[3]


def grid(nr, nc, seed):
    rng = np.random.default_rng(seed)
    lab = rng.permutation(nr * nc).reshape(nr, nc)
    ei = np.concatenate([lab[:, :-1].ravel(), lab[:-1, :].ravel()])
    ej = np.concatenate([lab[:, 1:].ravel(), lab[1:, :].ravel()])
    return lab, ei, ej


def test_grid_no_worse_than_strips():
    """A 32 x 32 grid with scattered labels, blocks of at most 64: strips of two rows cut
    15 x 32 = 480 edges, a random balanced partition about 15/16 of the 1984 edges; the
    partitioner does at least as well as the strips."""
    lab, ei, ej = grid(32, 32, 3)
    block, k, cut = cg.partition_columns(32 * 32, ei, ej, 64)
    check_valid(block, k, 1024, 64)
    strips = np.empty(1024, dtype=np.int64)
    for r in range(32):
        strips[lab[r]] = r // 2
    assert cut_of(strips, ei, ej) == 480
    rnd = np.random.default_rng(0).permutation(1024) // 64
    assert cut_of(rnd, ei, ej) > 1800
    assert cut <= 480


def planted(seed, q=512, c=32, p_in=0.3, p_out=0.002):
    rng = np.random.default_rng(seed)
    grp = rng.permutation(q) // c
    a, b = np.triu_indices(q, 1)
    keep = np.where(grp[a] == grp[b], rng.random(a.size) < p_in, rng.random(a.size) < p_out)
    return grp, a[keep], b[keep]


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_planted_partition_recovered(seed):
    """16 planted clusters of 32 columns, dense inside (p = 0.3) and sparse across
    (p = 0.002).  With blocks of up to 40 (or 64, two clusters a block) the cut is no
    worse than the planted one; with blocks of exactly the cluster size, where every block
    must be full, within 5 % of it."""
    grp, ei, ej = planted(seed)
    planted_cut = cut_of(grp, ei, ej)
    for cap in (40, 64):
        block, k, cut = cg.partition_columns(512, ei, ej, cap)
        check_valid(block, k, 512, cap)
        assert cut <= planted_cut
    block, k, cut = cg.partition_columns(512, ei, ej, 32)
    check_valid(block, k, 512, 32)
    assert cut <= 1.05 * planted_cut


def test_large_graph_is_quick():
    """q = 20000 columns (the largest configured output count), a chain with random links:
    well under a second on the host, and far below a random partition's cut."""
    import time
    rng = np.random.default_rng(7)
    q = 20000
    i = np.arange(q - 1)
    ei = np.concatenate([i, rng.integers(0, q, 20000)])
    ej = np.concatenate([i + 1, rng.integers(0, q, 20000)])
    t0 = time.perf_counter()
    block, k, cut = cg.partition_columns(q, ei, ej, 4096)
    assert time.perf_counter() - t0 < 5.0
    check_valid(block, k, q, 4096)
    rnd = np.random.default_rng(0).permutation(q) // 4096
    assert cut < 0.8 * cut_of(rnd, ei, ej)


def test_deterministic():
    ei, ej = er_graph(500, 3000, 9)
    r1 = cg.partition_columns(500, ei, ej, 50)
    r2 = cg.partition_columns(500, ei, ej, 50)
    assert np.array_equal(r1[0], r2[0]) and r1[1:] == r2[1:]


def row_blocks_of(block, ti, tj):
    return len(set(zip(np.asarray(ti).tolist(), block[np.asarray(tj)].tolist())))


def test_theta_partition_keeps_rows_in_one_block():
    """Columns in 12 scattered groups of 8; every row's active entries lie in one group.
    With blocks of 16 each row can touch a single block, so the cost Section 4.2
    minimises (rows x blocks touched) equals the number of non-empty rows."""
    rng = np.random.default_rng(5)
    p, q, c = 300, 96, 8
    groups = rng.permutation(q).reshape(-1, c)
    ti, tj = [], []
    for i in range(p):
        if i % 7 == 3:
            continue                                    # an empty row
        g = groups[rng.integers(len(groups))]
        cols = rng.choice(g, size=rng.integers(1, c + 1), replace=False)
        ti += [i] * len(cols)
        tj += cols.tolist()
    block, k, rb = cg.partition_theta_columns(p, q, ti, tj, 16)
    check_valid(block, k, q, 16)
    assert rb == row_blocks_of(block, ti, tj)
    assert rb == len(set(ti))


def test_theta_row_blocks_matches_definition_on_random_sets():
    rng = np.random.default_rng(6)
    for p, q, m, cap in [(50, 40, 300, 8), (200, 120, 2000, 32), (10, 5, 0, 2)]:
        ti = rng.integers(0, p, m)
        tj = rng.integers(0, q, m)
        block, k, rb = cg.partition_theta_columns(p, q, ti, tj, cap)
        check_valid(block, k, q, cap)
        assert rb == row_blocks_of(block, ti, tj)
        contiguous = np.arange(q) // cap
        assert rb <= row_blocks_of(contiguous, ti, tj) + p   # sanity: same order of cost


def test_theta_dense_rows_use_the_path_form():
    """Rows with more than 16 active columns join them as a path; a single full row over
    q columns then costs ceil(q / B) blocks, the least possible."""
    p, q = 3, 100
    ti = np.repeat(np.arange(p), q)
    tj = np.tile(np.arange(q), p)
    block, k, rb = cg.partition_theta_columns(p, q, ti, tj, 25)
    check_valid(block, k, q, 25)
    assert k == 4 and rb == 3 * 4


@pytest.mark.parametrize("args", [
    dict(q=-1, ei=[], ej=[], max_block=1),
    dict(q=3, ei=[0], ej=[3], max_block=1),
    dict(q=3, ei=[-1], ej=[0], max_block=1),
    dict(q=3, ei=[0], ej=[1], max_block=0),
    dict(q=3, ei=[0], ej=[1], max_block=2, w=[-1.0]),
    dict(q=3, ei=[0], ej=[1], max_block=2, w=[float("nan")]),
])
def test_bad_arguments_are_einval(args):
    with pytest.raises(cg.CGGMError):
        cg.partition_columns(**args)


def test_theta_bad_arguments_are_einval():
    with pytest.raises(cg.CGGMError):
        cg.partition_theta_columns(2, 3, [2], [0], 2)
    with pytest.raises(cg.CGGMError):
        cg.partition_theta_columns(2, 3, [0], [3], 2)
    with pytest.raises(cg.CGGMError):
        cg.partition_theta_columns(2, 3, [0], [1], 0)
