"""Host arithmetic of the server's admission rule (no GPU): cggm_footprint, the device bytes
a request is accounted for."""
import itertools

import paper_1509_04681_gb300 as cg

HBM_BYTES = 284_208 * 2**20     # one GB300


def test_invalid_sizes():
    for n, p, q in [(0, 1, 1), (1, 0, 1), (1, 1, 0), (-5, 10, 10)]:
        assert cg.footprint(n, p, q) == -1


def test_monotone_in_every_size():
    sizes = [1, 7, 64, 500, 3000]
    for prec in (cg.CGGM_FP64, cg.CGGM_MIXED):
        for n, p, q in itertools.product(sizes, repeat=3):
            f = cg.footprint(n, p, q, prec)
            assert f > 0
            assert cg.footprint(2 * n, p, q, prec) >= f
            assert cg.footprint(n, 2 * p, q, prec) >= f
            assert cg.footprint(n, p, 2 * q, prec) >= f


def test_covers_the_double_precision_state():
    """At least the double q x q matrices (S_yy, Lambda, its factor, Sigma, G_Lambda, D) and
    p x q matrices (S_xy, Theta, G_Theta) and the transposed X, Y that a solve keeps."""
    for n, p, q in [(1000, 5000, 5000), (500, 40000, 20000), (100, 200, 100)]:
        floor = 8 * (6 * q * q + 3 * p * q + n * (p + q))
        for prec in (cg.CGGM_FP64, cg.CGGM_MIXED):
            assert cg.footprint(n, p, q, prec) >= floor


def test_largest_configured_workload_fits_one_gpu():
    """p = 40000, q = 20000, n = 500: one solve fits in a GB300's memory."""
    for prec in (cg.CGGM_FP64, cg.CGGM_MIXED):
        assert cg.footprint(500, 40000, 20000, prec) < 0.5 * HBM_BYTES


def test_sxx_is_held_in_chunks_of_at_most_256_mib():
    """Only up to 256 MiB of S_xx rows count at large p: doubling p from 40000 to 80000
    adds far less than the 19 GB a whole double S_xx would."""
    for prec in (cg.CGGM_FP64, cg.CGGM_MIXED):
        a = cg.footprint(500, 40000, 20000, prec)
        b = cg.footprint(500, 80000, 20000, prec)
        per_pq = 8 * 6 + 4  # the p x q matrices a solve keeps, double and cache type
        assert b - a < per_pq * 40000 * 20000 * 1.2 + (1 << 30)
