"""Pins of the oracle's negacyclic product, gadget decomposition and modulus
switch against brute force, closed forms and exact rational arithmetic."""
import random
from fractions import Fraction

import numpy as np
import pytest

M32 = 1 << 32


def brute_negacyclic(a, b):
    """Full product with Python integers, then X^N = -1, then mod 2^32."""
    N = len(a)
    full = [0] * (2 * N - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            full[i + j] += int(x) * int(y)
    red = [full[k] - (full[k + N] if k + N < 2 * N - 1 else 0) for k in range(N)]
    return [v % M32 for v in red]


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_negacyclic_brute_force(O, N):
    rng = np.random.default_rng(N)
    for _ in range(20):
        a = rng.integers(0, M32, N, dtype=np.uint64).astype(np.uint32)
        b = rng.integers(0, M32, N, dtype=np.uint64).astype(np.uint32)
        assert list(O.poly_mul(a, b)) == brute_negacyclic(a, b)


def xk(N, k):
    """The monomial X^k (k in [0, 2N)) as a uint32 polynomial."""
    p = np.zeros(N, np.uint32)
    p[k % N] = 1 if k < N else M32 - 1
    return p


def test_negacyclic_closed_forms_full_size(O):
    N = 1024
    rng = np.random.default_rng(1)
    a = rng.integers(0, M32, N, dtype=np.uint64).astype(np.uint32)
    b = rng.integers(0, M32, N, dtype=np.uint64).astype(np.uint32)
    c = rng.integers(0, M32, N, dtype=np.uint64).astype(np.uint32)
    one = xk(N, 0)
    assert (O.poly_mul(a, one) == a).all()
    assert (O.poly_mul(a, xk(N, N)) == (-a.astype(np.int64) % M32)).all()  # X^N = -1
    for k in (1, 7, 500, 1023, 1024 + 3):
        kk = k % N
        sign = 1 if k < N else -1
        rolled = np.roll(a.astype(np.int64), kk)
        rolled[:kk] = -rolled[:kk]          # wrapped coefficients change sign
        assert (O.poly_mul(a, xk(N, k)) == (sign * rolled) % M32).all()
    # commutativity and distributivity
    assert (O.poly_mul(a, b) == O.poly_mul(b, a)).all()
    lhs = O.poly_mul(a, (b.astype(np.uint64) + c) % M32)
    rhs = (O.poly_mul(a, b).astype(np.uint64) + O.poly_mul(a, c)) % M32
    assert (lhs == rhs).all()


def independent_digits(x, l=3, Bgbit=10):
    """Signed base-2^Bgbit digits of x rounded to l*Bgbit bits, computed
    least-significant first by centered remainders (a different algorithm
    from the oracle's offset method)."""
    drop = 32 - l * Bgbit
    v = ((x + (1 << (drop - 1))) % M32) >> drop if drop else x
    B = 1 << Bgbit
    out = []
    for _ in range(l):
        d = v % B
        if d >= B // 2:
            d -= B
        out.append(d)
        v = (v - d) // B
    return out[::-1]  # most significant first


def test_decompose_recomposition_and_range(O):
    p = O.GATE_PARAMS
    rng = random.Random(5)
    edge = [0, 1, 2, 3, 4, 5, 6, 2 ** 31, 2 ** 31 - 1, 2 ** 31 + 2, M32 - 1, M32 - 2, M32 - 3,
            2 ** 21, 2 ** 21 - 2, 2 ** 11 - 2, 2 ** 30, 3 * 2 ** 30 + 2]
    vals = edge + [rng.randrange(M32) for _ in range(20000)]
    for x in vals:
        d = O.decompose(p, x)
        assert all(-512 <= v <= 511 for v in d), (x, d)
        rounded = ((x + 2) // 4 * 4) % M32
        assert sum(v << (32 - 10 * (i + 1)) for i, v in enumerate(d)) % M32 == rounded, x
        assert d == independent_digits(x), x


def test_decompose_other_bases(O):
    for l, Bgbit in ((2, 8), (4, 6), (1, 16)):
        p = O.Params(l=l, Bgbit=Bgbit)
        rng = random.Random(l)
        for _ in range(2000):
            x = rng.randrange(M32)
            assert O.decompose(p, x) == independent_digits(x, l, Bgbit)


def test_modswitch_exact_rounding(O):
    rng = random.Random(9)
    for N in (1024, 64):
        twoN = 2 * N
        step = M32 // twoN
        vals = [0, M32 - 1, step // 2, step // 2 - 1, 3 * step + step // 2, 7 * step + step // 2 - 1]
        vals += [rng.randrange(M32) for _ in range(5000)]
        for x in vals:
            exact = Fraction(x * twoN, M32) + Fraction(1, 2)
            assert O.modswitch(x, N) == (exact.numerator // exact.denominator) % twoN, (x, N)
