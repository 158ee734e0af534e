"""The seeded input generators (CPU): each property the input recipe states is checked
against its definition or a closed form, so that the workloads are what the design notes
say they are.  The generators hold none of the method's arithmetic."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import synth


def test_streams_reproducible_and_independent():
    a = synth.make_problem(30, 12, 40, lam_kind="chain", seed=3)
    b = synth.make_problem(30, 12, 40, lam_kind="chain", seed=3)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y)
    assert (a.Theta_true != b.Theta_true).nnz == 0
    c = synth.make_problem(30, 12, 40, lam_kind="chain", seed=4)
    assert not np.array_equal(a.X, c.X)
    # X and Theta come from their own streams: changing the network leaves them as they are
    d = synth.make_problem(30, 12, 40, lam_kind="random3", seed=3)
    assert np.array_equal(a.X, d.X)
    assert (a.Theta_true != d.Theta_true).nnz == 0
    assert not np.array_equal(a.Y, d.Y)


@pytest.mark.parametrize("q", [1, 2, 7, 50])
def test_chain_precision_spectrum(q):
    """Tridiagonal Toeplitz: eigenvalues 1 + 0.8 cos(k pi / (q + 1)), k = 1..q."""
    L = synth.chain_precision(q).toarray()
    assert np.all(np.diag(L) == 1.0)
    if q > 1:
        assert np.all(np.diag(L, 1) == 0.4) and np.all(np.diag(L, -1) == 0.4)
        assert np.count_nonzero(L) == q + 2 * (q - 1)
    k = np.arange(1, q + 1)
    ev = np.sort(1.0 + 0.8 * np.cos(k * np.pi / (q + 1))) if q > 1 else np.array([1.0])
    assert np.allclose(np.linalg.eigvalsh(L), ev, atol=1e-12)


@pytest.mark.parametrize("q,d", [(200, 4.0), (57, 3.0), (10, 0.0)])
def test_random_sparse_precision(q, d):
    rng = np.random.default_rng(q)
    L = synth.random_sparse_precision(q, d, rng).toarray()
    assert np.array_equal(L, L.T)
    off = L - np.diag(np.diag(L))
    assert np.count_nonzero(off) == 2 * int(round(q * d / 2))     # distinct edges, both halves
    w = np.abs(off[off != 0])
    assert np.all((w >= 0.2) & (w <= 0.5))
    rowsum = np.abs(off).sum(axis=1)
    assert np.allclose(np.diag(L), np.maximum(1.0, rowsum + 0.2), rtol=0, atol=1e-15)
    # strict diagonal dominance by 0.2: Gershgorin bounds every eigenvalue below by 0.2
    assert np.linalg.eigvalsh(L).min() >= 0.2 - 1e-12


def test_random_links_added_to_a_chain_keep_it():
    rng = np.random.default_rng(0)
    base = synth.chain_precision(40)
    L = synth.random_sparse_precision(40, 2.0, rng, base=base).toarray()
    assert np.all(np.diag(L, 1) == 0.4)
    assert np.count_nonzero(L - np.diag(np.diag(L))) == 2 * (39 + 40)


def test_sparse_theta_columns():
    rng = np.random.default_rng(1)
    T = synth.sparse_theta(50, 30, 5, rng)
    assert T.shape == (50, 30)
    cnt = np.diff(T.tocsc().indptr)
    assert np.all(cnt == 5)
    v = np.abs(T.data)
    assert np.all((v >= 0.5) & (v <= 1.0))
    assert np.any(T.data < 0) and np.any(T.data > 0)


def test_genotype_inputs():
    rng = np.random.default_rng(2)
    n, p = 2000, 300
    X, raw = synth.genotype_X(n, p, rng, return_raw=True)
    assert raw.dtype == np.int8 and set(np.unique(raw).tolist()) <= {0, 1, 2}
    assert np.all(raw.min(axis=0) < raw.max(axis=0))                   # no constant column
    assert np.unique(raw.T, axis=0).shape[0] == p                       # no duplicate column
    # standardised with the population sd: zero mean, (X^T X / n)_kk = 1
    assert np.max(np.abs(X.mean(axis=0))) < 1e-12
    assert np.allclose(np.einsum("ij,ij->j", X, X) / n, 1.0, atol=1e-12)
    # it is raw standardised
    mu, sd = raw.mean(axis=0), raw.astype(float).std(axis=0)
    assert np.allclose(X, (raw - mu) / sd, atol=1e-12)
    # allele frequencies from MAF ~ U(0.05, 0.5): with 2n alleles, within a few percent
    freq = raw.mean(axis=0) / 2.0
    assert freq.min() > 0.02 and freq.max() < 0.56


def test_outputs_follow_the_model():
    """Y = -X Theta Sigma + E with rows of E ~ N(0, Sigma), Sigma = Lambda^-1: for many
    samples the residual has mean 0 and covariance Sigma, and the regression of Y on X
    recovers -Theta Sigma."""
    rng = np.random.default_rng(3)
    n, p, q = 40000, 3, 4
    X = rng.standard_normal((n, p))
    Theta = sp.csc_matrix(np.array([[0.8, 0, 0, -0.6], [0, 0.7, 0, 0], [0, 0, -0.9, 0.5]]))
    Lam = synth.chain_precision(q)
    Sigma = np.linalg.inv(Lam.toarray())
    Y = synth.sample_Y(X, Theta, Lam, rng)
    B = -Theta.toarray() @ Sigma
    E = Y - X @ B
    assert np.max(np.abs(E.mean(axis=0))) < 0.03
    C = E.T @ E / n
    assert np.max(np.abs(C - Sigma)) < 0.05 * np.max(np.abs(Sigma))
    B_hat = np.linalg.lstsq(X, Y, rcond=None)[0]
    assert np.max(np.abs(B_hat - B)) < 0.03


def test_named_workloads():
    W = synth.WORKLOADS
    assert {k: (v["p"], v["q"], v["n"]) for k, v in W.items()} == {
        "chain-gauss-p200-q100-n100": (200, 100, 100),
        "chain-geno-p5000-q5000-n1000": (5000, 5000, 1000),
        "rand4-geno-p40000-q20000-n500": (40000, 20000, 500),
    }
    pr = synth.workload("chain-gauss-p200-q100-n100")
    assert pr.X.shape == (100, 200) and pr.Y.shape == (100, 100) and pr.lam_L == 0.1


def test_serving_requests():
    """Sizes log-uniform in the ranges (here divided by 4, as the served benchmark uses
    them), an 8-point geometric grid from 0.5 to 0.02, Poisson arrivals at 20/s."""
    reqs = synth.serving_requests(n_req=400, rate_per_s=20.0, seed=0, p_range=(125, 2000),
                                  q_range=(50, 1000), n_range=(50, 250))
    assert all(125 <= r.p <= 2000 and 50 <= r.q <= 1000 and 50 <= r.n <= 250 for r in reqs)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 15.0 < len(reqs) / t[-1] < 25.0
    g = reqs[0].lambdas
    assert len(g) == 8 and g[0] == 0.5 and abs(g[-1] - 0.02) < 1e-15
    ratios = np.array(g[1:]) / np.array(g[:-1])
    assert np.allclose(ratios, 0.04 ** (1 / 7), rtol=1e-12)
    kinds = {r.lam_kind for r in reqs}
    assert kinds == {"chain", "random4"}
    # log-uniform: the median size sits near the geometric mean of its range
    assert abs(math.log(np.median([r.p for r in reqs])) - math.log(math.sqrt(125 * 2000))) < 0.3


def test_clustered_family_recipe():
    """The paper's random graphs with clustering (Section 5): clusters of 250, average degree
    10, 90 % of edges inside clusters, unit weights, Lambda positive definite; Theta with
    round(100 sqrt(p)) active inputs (at most p) and 10 q unit edges."""
    import math
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    q = 1000
    L = synth.clustered_precision(q, rng)
    assert (abs(L - L.T) > 0).nnz == 0
    off = sp.triu(L, k=1).tocoo()
    assert off.nnz == q * 10 // 2
    assert np.all(off.data == 1.0)
    intra = np.mean(off.row // 250 == off.col // 250)
    assert abs(intra - 0.9) < 0.01
    deg = np.asarray((L != 0).sum(axis=1)).ravel() - 1
    assert abs(deg.mean() - 10.0) < 1e-9
    assert np.linalg.eigvalsh(L.toarray()).min() > 0.09
    p = 4000
    T = synth.clustered_theta(p, q, rng)
    assert T.nnz == 10 * q and np.all(T.data == 1.0)
    assert np.unique(T.tocoo().row).size == min(p, round(100 * math.sqrt(p)))  # all 4000
    T2 = synth.clustered_theta(1_000_000, q, rng)   # 100 sqrt(p) = 10^5 > 10 q: capped at 10 q
    assert T2.nnz == 10 * q and np.unique(T2.tocoo().row).size == 10 * q
    T3 = synth.clustered_theta(90_000, 5000, rng)   # 30000 chosen inputs, 50000 edges
    assert T3.nnz == 50_000 and np.unique(T3.tocoo().row).size == 30_000
    small = synth.clustered_theta(50, 20, rng)   # 100 sqrt(50) > 50: every input may be used
    assert small.nnz == 200
    pr = synth.clustered_problem(300, 300, seed=1)
    assert pr.X.shape == (200, 300) and pr.Y.shape == (200, 300)
