"""Seeded generators for the synthetic CGGM workloads.

Every array is drawn from its own PCG64 stream, spawned from one integer seed in a
fixed order, so that a (workload, seed) pair names the same bytes on every machine:

    stream 0: X                 stream 2: Theta support, signs and magnitudes
    stream 1: Lambda structure  stream 3: the noise Z of Y

The model is the CGGM of Section 2.1.  Its negative log-likelihood (Eq. 1) is that of
y | x ~ N(-Lambda^-1 Theta^T x, Lambda^-1); in row-sample form Y = -X Theta Sigma + E with
Sigma = Lambda^-1 and each row of E drawn from N(0, Sigma).  The chain graph follows the
synthetic experiments of Section 5.1 (tridiagonal Lambda, one output per input chain);
the diagonal and off-diagonal values, the Theta values and the genotype-like inputs
are those of the workloads this library is measured on.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

STREAM_X, STREAM_LAMBDA, STREAM_THETA, STREAM_NOISE = 0, 1, 2, 3
N_STREAMS = 4


def _streams(seed: int):
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(N_STREAMS)]


def chain_precision(q: int, diag: float = 1.0, off: float = 0.4) -> sp.csr_matrix:
    """Tridiagonal chain precision matrix (q x q): Lambda_ii = diag, Lambda_{i,i+-1} = off.

    With diag = 1 and |off| < 1/2 every eigenvalue (diag + 2 off cos(k pi/(q+1))) is
    positive, so the matrix is positive definite."""
    if q == 1:
        return sp.csr_matrix(np.array([[diag]]))
    d = np.full(q, diag)
    o = np.full(q - 1, off)
    return sp.diags([o, d, o], [-1, 0, 1], format="csr")


def random_sparse_precision(q: int, avg_degree: float, rng: np.random.Generator,
                            lo: float = 0.2, hi: float = 0.5, margin: float = 0.2,
                            base: Optional[sp.csr_matrix] = None) -> sp.csr_matrix:
    """Random sparse, strictly diagonally dominant precision matrix.

    q*avg_degree/2 distinct undirected edges are drawn uniformly; each gets a weight
    of random sign and magnitude U(lo, hi).  If ``base`` is given its off-diagonal
    entries are kept and the random links are added to it.  The diagonal is set to
    max(1, sum_j |Lambda_ij| + margin), so Lambda is symmetric positive definite."""
    n_edges = int(round(q * avg_degree / 2.0))
    rows, cols, vals = [], [], []
    if base is not None:
        b = sp.triu(base, k=1).tocoo()
        rows.append(b.row); cols.append(b.col); vals.append(b.data)
    if n_edges > 0 and q > 1:
        # Draw with replacement, then drop self loops and duplicates; top up until done.
        seen = set()
        if base is not None:
            seen.update(zip(rows[0].tolist(), cols[0].tolist()))
        er, ec = [], []
        while len(er) < n_edges:
            need = n_edges - len(er)
            a = rng.integers(0, q, size=2 * need + 16)
            b2 = rng.integers(0, q, size=2 * need + 16)
            for i, j in zip(a.tolist(), b2.tolist()):
                if i == j:
                    continue
                i, j = (i, j) if i < j else (j, i)
                if (i, j) in seen:
                    continue
                seen.add((i, j))
                er.append(i); ec.append(j)
                if len(er) == n_edges:
                    break
        w = rng.uniform(lo, hi, size=len(er)) * rng.choice([-1.0, 1.0], size=len(er))
        rows.append(np.asarray(er)); cols.append(np.asarray(ec)); vals.append(w)
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    v = np.concatenate(vals) if vals else np.zeros(0)
    upper = sp.coo_matrix((v, (r, c)), shape=(q, q))
    off = (upper + upper.T).tocsr()
    rowsum = np.asarray(abs(off).sum(axis=1)).ravel()
    diag = np.maximum(1.0, rowsum + margin)
    return (off + sp.diags(diag)).tocsr()


def sparse_theta(p: int, q: int, nnz_per_col: int, rng: np.random.Generator,
                 lo: float = 0.5, hi: float = 1.0) -> sp.csc_matrix:
    """p x q Theta with ``nnz_per_col`` nonzeros per column at distinct random rows,
    values of random sign and magnitude U(lo, hi)."""
    k = min(nnz_per_col, p)
    rows = np.concatenate([rng.choice(p, size=k, replace=False) for _ in range(q)]) \
        if k > 0 else np.zeros(0, dtype=np.int64)
    cols = np.repeat(np.arange(q), k)
    vals = rng.uniform(lo, hi, size=rows.size) * rng.choice([-1.0, 1.0], size=rows.size)
    return sp.csc_matrix((vals, (rows, cols)), shape=(p, q))


def gaussian_X(n: int, p: int, rng: np.random.Generator) -> np.ndarray:
    """n x p inputs, iid N(0, 1), float64, row-major."""
    return rng.standard_normal((n, p))


def genotype_X(n: int, p: int, rng: np.random.Generator, standardise: bool = True,
               return_raw: bool = False):
    """Genotype-like inputs: X_raw[s, k] ~ Binomial(2, MAF_k), MAF_k ~ U(0.05, 0.5).

    Columns that come out constant, or equal to an earlier column, are redrawn (a
    constant column has no standardisation; duplicates make Theta non-identifiable).
    With ``standardise`` each column is centred and divided by its population
    standard deviation (1/n), so that (X^T X / n)_kk = 1.  Returns float64 X (and the
    int8 raw genotypes with ``return_raw``)."""
    maf = rng.uniform(0.05, 0.5, size=p)
    raw = rng.binomial(2, maf[None, :], size=(n, p)).astype(np.int8)
    for _ in range(100):
        bad = np.flatnonzero(raw.min(axis=0) == raw.max(axis=0))
        if n <= 4096 and p <= 20000:
            # duplicate columns (only plausible for small n)
            _, first = np.unique(raw.T, axis=0, return_index=True)
            dup = np.setdiff1d(np.arange(p), first)
            bad = np.union1d(bad, dup)
        if bad.size == 0:
            break
        raw[:, bad] = rng.binomial(2, maf[None, bad], size=(n, bad.size)).astype(np.int8)
    X = raw.astype(np.float64)
    if standardise:
        mu = X.mean(axis=0)
        sd = X.std(axis=0)
        X = (X - mu) / sd
    return (X, raw) if return_raw else X


def sample_Y(X: np.ndarray, Theta: sp.spmatrix, Lambda: sp.spmatrix,
             rng: np.random.Generator) -> np.ndarray:
    """Y = -X Theta Lambda^-1 + E, rows of E ~ N(0, Lambda^-1) (Eq. 1's model).

    With Lambda = L L^T (Cholesky), e = L^-T z for z ~ N(0, I) has covariance
    L^-T L^-1 = Lambda^-1.  Dense Cholesky (q up to a few 10^4)."""
    n = X.shape[0]
    q = Lambda.shape[0]
    Ld = Lambda.toarray() if sp.issparse(Lambda) else np.asarray(Lambda)
    L = np.linalg.cholesky(Ld)
    XT = np.asarray((sp.csr_matrix(X) @ Theta).todense()) if sp.issparse(X) else \
        np.asarray(Theta.T @ X.T).T
    Z = rng.standard_normal((n, q))
    mean = -sla.cho_solve((L, True), XT.T).T
    E = sla.solve_triangular(L, Z.T, lower=True, trans="T").T
    return mean + E


def clustered_precision(q: int, rng: np.random.Generator, cluster: int = 250,
                        avg_degree: float = 10.0, intra: float = 0.9,
                        margin: float = 0.1) -> sp.csr_matrix:
    """The clustered random network of the paper's second synthetic family (Section 5):
    outputs in consecutive clusters of ``cluster`` nodes (the last one may be smaller),
    q * avg_degree / 2 distinct edges of weight 1, a fraction ``intra`` of them between two
    random nodes of one cluster (the cluster drawn in proportion to its number of node pairs)
    and the rest between two random nodes anywhere.  The paper sets the diagonal so that
    Lambda is positive definite; here it is the row's absolute sum plus ``margin`` (strictly
    diagonally dominant)."""
    n_edges = int(round(q * avg_degree / 2.0))
    starts = np.arange(0, q, cluster)
    sizes = np.minimum(cluster, q - starts)
    pairs = sizes * (sizes - 1) / 2.0
    n_pairs_all = q * (q - 1) / 2.0
    n_intra = min(int(round(intra * n_edges)), int(pairs.sum()))
    n_inter = min(n_edges - n_intra, int(n_pairs_all - pairs.sum()))
    seen = set()
    rows, cols = [], []

    def add(i, j):
        i, j = (i, j) if i < j else (j, i)
        if i == j or (i, j) in seen:
            return False
        seen.add((i, j))
        rows.append(i)
        cols.append(j)
        return True

    prob = pairs / pairs.sum() if pairs.sum() > 0 else None
    k = 0
    while k < n_intra:
        c = rng.choice(len(sizes), p=prob)
        a, b = rng.integers(0, sizes[c], size=2)
        if add(starts[c] + a, starts[c] + b):
            k += 1
    cid = np.repeat(np.arange(len(sizes)), sizes)
    k = 0
    while k < n_inter:
        a, b = rng.integers(0, q, size=2)
        if cid[a] != cid[b] and add(a, b):
            k += 1
    r = np.asarray(rows, dtype=np.int64)
    c = np.asarray(cols, dtype=np.int64)
    upper = sp.coo_matrix((np.ones(r.size), (r, c)), shape=(q, q))
    off = (upper + upper.T).tocsr()
    diag = np.asarray(abs(off).sum(axis=1)).ravel() + margin
    return (off + sp.diags(diag)).tocsr()


def clustered_theta(p: int, q: int, rng: np.random.Generator, inputs: Optional[int] = None,
                    edges_per_output: int = 10) -> sp.csc_matrix:
    """Theta of the clustered family (Section 5): min(p, round(100 sqrt(p))) inputs chosen at
    random have edges to at least one output; edges_per_output * q distinct edges of weight 1
    in all: one from each chosen input to a random output, the rest from random chosen inputs
    to random outputs."""
    total_want = edges_per_output * q
    k = min(p, int(round(100.0 * math.sqrt(p)))) if inputs is None else min(p, inputs)
    k = min(k, total_want)  # every chosen input keeps an edge
    sel = rng.choice(p, size=k, replace=False)
    total = min(total_want, k * q)
    seen = set()
    rows, cols = [], []
    for i in sel.tolist():
        j = int(rng.integers(0, q))
        seen.add((i, j))
        rows.append(i)
        cols.append(j)
    while len(rows) < total:
        i = int(sel[rng.integers(0, k)])
        j = int(rng.integers(0, q))
        if (i, j) in seen:
            continue
        seen.add((i, j))
        rows.append(i)
        cols.append(j)
    return sp.csc_matrix((np.ones(len(rows)), (rows, cols)), shape=(p, q))


def clustered_problem(p: int, q: int, n: int = 200, lam: float = 0.1, seed: int = 0,
                      name: Optional[str] = None) -> "Problem":
    """The paper's random graphs with clustering (Section 5): clustered Lambda, Theta on
    100 sqrt(p) inputs with 10 q edges, Gaussian inputs X ~ N(0, 1) (the paper does not state
    their distribution), Y drawn from the CGGM; n = 200 as in the paper."""
    sx, sl, st, sn = _streams(seed)
    X = gaussian_X(n, p, sx)
    Lam = clustered_precision(q, sl)
    Th = clustered_theta(p, q, st)
    Y = sample_Y(X, Th, Lam, sn)
    return Problem(name=name or f"cluster-gauss-p{p}-q{q}-n{n}", X=X, Y=Y, Lambda_true=Lam,
                   Theta_true=Th, lam_L=lam, lam_T=lam, seed=seed)


@dataclasses.dataclass
class Problem:
    name: str
    X: np.ndarray               # n x p float64, row-major
    Y: np.ndarray               # n x q float64, row-major
    Lambda_true: sp.csr_matrix  # q x q
    Theta_true: sp.csc_matrix   # p x q
    lam_L: float
    lam_T: float
    seed: int
    X_raw: Optional[np.ndarray] = None  # int8 genotypes when x_kind == "genotype"

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def p(self):
        return self.X.shape[1]

    @property
    def q(self):
        return self.Y.shape[1]


# Workloads, named by what they are and their sizes.
WORKLOADS = {
    # plain single solve, Gaussian inputs
    "chain-gauss-p200-q100-n100": dict(p=200, q=100, n=100, x_kind="gaussian",
                                       lam_kind="chain", theta_nnz=5, lam=0.1, seed=0),
    # genotype-like inputs, chain network: the mixed-vs-FP64 single solve
    "chain-geno-p5000-q5000-n1000": dict(p=5000, q=5000, n=1000, x_kind="genotype",
                                         lam_kind="chain", theta_nnz=10, lam=0.05, seed=0),
    # large single solve, random sparse network of average degree 4
    "rand4-geno-p40000-q20000-n500": dict(p=40000, q=20000, n=500, x_kind="genotype",
                                          lam_kind="random4", theta_nnz=20, lam=0.1, seed=0),
}


def make_problem(p: int, q: int, n: int, x_kind: str = "gaussian", lam_kind: str = "chain",
                 theta_nnz: int = 5, lam: float = 0.1, seed: int = 0,
                 name: Optional[str] = None) -> Problem:
    """Draw one problem.  ``x_kind`` in {gaussian, genotype}; ``lam_kind`` in
    {chain, random4, random<d>}; ``theta_nnz`` nonzeros per column of the true Theta."""
    sx, sl, st, sn = _streams(seed)
    raw = None
    if x_kind == "gaussian":
        X = gaussian_X(n, p, sx)
    elif x_kind == "genotype":
        X, raw = genotype_X(n, p, sx, return_raw=True)
    else:
        raise ValueError(f"unknown x_kind {x_kind!r}")
    if lam_kind == "chain":
        Lam = chain_precision(q)
    elif lam_kind.startswith("random"):
        Lam = random_sparse_precision(q, float(lam_kind[len("random"):]), sl)
    else:
        raise ValueError(f"unknown lam_kind {lam_kind!r}")
    Th = sparse_theta(p, q, theta_nnz, st)
    Y = sample_Y(X, Th, Lam, sn)
    return Problem(name=name or f"{lam_kind}-{x_kind}-p{p}-q{q}-n{n}", X=X, Y=Y,
                   Lambda_true=Lam, Theta_true=Th, lam_L=lam, lam_T=lam, seed=seed, X_raw=raw)


def workload(name: str, **overrides) -> Problem:
    cfg = dict(WORKLOADS[name])
    cfg.update(overrides)
    return make_problem(name=name, **cfg)


@dataclasses.dataclass
class ServingRequest:
    rid: int
    arrival_s: float
    p: int
    q: int
    n: int
    lam_kind: str
    lambdas: tuple
    seed: int

    def problem(self) -> Problem:
        return make_problem(self.p, self.q, self.n, x_kind="gaussian", lam_kind=self.lam_kind,
                            theta_nnz=5, lam=self.lambdas[0], seed=self.seed,
                            name=f"req{self.rid}")


def serving_requests(n_req: int = 64, rate_per_s: float = 20.0, seed: int = 0,
                     p_range=(500, 8000), q_range=(200, 4000), n_range=(200, 1000),
                     n_lambda: int = 8, lam_hi: float = 0.5, lam_lo: float = 0.02):
    """Regularisation-path requests of uneven size arriving as a Poisson process.

    Sizes are log-uniform in the given ranges; each request carries an ``n_lambda``
    point geometric grid from lam_hi down to lam_lo (lambda_Lambda = lambda_Theta);
    Lambda is a chain or a random sparse graph of average degree 4 with probability
    1/2 each; gaps between arrivals are exponential with mean 1/rate."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed).spawn(1)[0]))

    def logu(lo, hi):
        return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))

    grid = tuple(float(lam_hi * (lam_lo / lam_hi) ** (k / (n_lambda - 1)))
                 for k in range(n_lambda))
    t = 0.0
    out = []
    for r in range(n_req):
        t += rng.exponential(1.0 / rate_per_s)
        out.append(ServingRequest(rid=r, arrival_s=t, p=logu(*p_range), q=logu(*q_range),
                                  n=logu(*n_range),
                                  lam_kind="chain" if rng.uniform() < 0.5 else "random4",
                                  lambdas=grid, seed=int(1000 + r)))
    return out
