"""Pins of the oracle's random sources (PRNG, Gaussian, key bits)."""
import math
import os

import numpy as np

from conftest import signed32

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def test_splitmix64_published_vector(O):
    lines = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    seed = int(lines[0][1])
    expected = [int(ln[0]) for ln in lines[1:]]
    assert [O.splitmix64_at(seed, k) for k in range(len(expected))] == expected


def test_uniform32_is_high_half_of_domain_segment(O):
    # domain d, index i is output d*2^40 + i of the seeded stream
    for d in (1, 5, 8):
        for i in (0, 1, 12345):
            assert O.uniform32(99, d, i) == O.splitmix64_at(99, (d << 40) + i) >> 32


def test_uniform32_bits_balanced(O):
    vals = np.array([O.uniform32(3, 7, i) for i in range(20000)], dtype=np.uint64)
    for b in (0, 15, 31):
        frac = ((vals >> b) & 1).mean()
        assert abs(frac - 0.5) < 5 * 0.5 / math.sqrt(len(vals))


def test_gauss_statistics(O):
    sigma = 2.0 ** -15
    n = 20000
    e = signed32([O.gauss32(11, 4, i, sigma) for i in range(n)]).astype(np.float64) / 2 ** 32
    # mean within 5 standard errors, variance within 5 standard errors of sigma^2
    assert abs(e.mean()) < 5 * sigma / math.sqrt(n)
    var = e.var()
    assert abs(var / sigma ** 2 - 1.0) < 5 * math.sqrt(2.0 / n)
    # Gaussian fourth moment: kurtosis 3
    k = ((e - e.mean()) ** 4).mean() / var ** 2
    assert abs(k - 3.0) < 0.25


def test_gauss_zero_sigma_is_exactly_zero(O):
    assert all(O.gauss32(5, 4, i, 0.0) == 0 for i in range(100))


def test_secret_key_bits(O):
    p = O.GATE_PARAMS
    s, K = O.secret_keygen(p, 2021)
    assert set(np.unique(s)) <= {0, 1} and set(np.unique(K)) <= {0, 1}
    assert 0.4 < s.mean() < 0.6 and 0.45 < K.mean() < 0.55
    s2, _ = O.secret_keygen(p, 2022)
    assert (s != s2).any()
