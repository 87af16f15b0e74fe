"""The algebra of the tensor-core external product, checked on the CPU.

The GPU's Toeplitz form (blind rotation's CMux products, §3 "TFHE Library")
rests on four facts, each checked here against the oracle's schoolbook
negacyclic product or against exact integers:

1. with the digit coefficients reversed (k = N - 1 - j), the negacyclic
   Toeplitz matrix of a key polynomial is the Hankel matrix f(n + k),
   f(s) = bt[s - (N - 1)], bt[s] = b[s] (s >= 0), -b[s + N] (s < 0);
2. an 8 x 8 core matrix stored as CM_q[r][c] = f(8q + r + c) and walked with
   equal strides in both dimensions reproduces every 128 x 16 operand tile;
3. balanced byte limbs of the key and balanced 5-bit limbs of the digits
   recombine exactly mod 2^32 and stay within |limb| <= 128 and <= 16;
4. fp32 accumulation of 6 x 1024 such limb products is exact, even in the
   worst case (every product at its maximum magnitude, one sign).
This is a model of the method, not of the CUDA code (whose parity against the
oracle is tested on the GPU).
"""
import numpy as np
import pytest

from oracle import oracle as O


def balanced_byte_limbs(x):
    """x (uint32 values) = sum_a 2^(8a) limb_a mod 2^32, limb_a in [-128, 127]."""
    x = np.asarray(x, dtype=np.int64) & 0xFFFFFFFF
    limbs = []
    for _ in range(4):
        l = ((x + 128) & 255) - 128
        limbs.append(l)
        x = ((x - l) & 0xFFFFFFFF) >> 8
    return limbs


def balanced_digit_limbs(d):
    """d in [-512, 511] = lo + 32 hi, lo in [-16, 15], hi in [-16, 16]."""
    d = np.asarray(d, dtype=np.int64)
    lo = ((d + 16) & 31) - 16
    return lo, (d - lo) >> 5


def hankel_f(b):
    N = len(b)
    s = np.arange(2 * N - 1)
    j = s - (N - 1)
    b = np.asarray(b, dtype=np.int64)
    return np.where(j >= 0, b[np.clip(j, 0, N - 1)], (-b[np.clip(j + N, 0, N - 1)]) & 0xFFFFFFFF)


def toeplitz_form_product(d, b, accumulate=np.float32):
    """The tensor form of the negacyclic product d * b mod 2^32."""
    N = len(b)
    f = hankel_f(b)
    n = np.arange(N)[:, None]
    k = np.arange(N)[None, :]
    dr = np.asarray(d, dtype=np.int64)[::-1]           # reversed digit coefficients
    total = np.zeros(N, dtype=np.int64)
    for a, fl in enumerate(balanced_byte_limbs(f)):
        H = fl[n + k]                                    # Hankel: depends on n + k only
        for bb, dl in enumerate(balanced_digit_limbs(dr)):
            S = (H.astype(accumulate) @ dl.astype(accumulate)).astype(np.int64)
            assert np.array_equal(S, H @ dl)             # the float sums are exact
            total = (total + ((S & 0xFFFFFFFF) << (8 * a + 5 * bb))) & 0xFFFFFFFF
    return total.astype(np.uint32)


@pytest.mark.parametrize("N", [16, 64, 1024])
def test_toeplitz_form_equals_negacyclic_product(N):
    rng = np.random.default_rng(N)
    for trial in range(3):
        b = rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32)
        d = rng.integers(-512, 512, N)
        if trial == 1:
            b[:] = 0x80000000                            # extreme key words
            d[:] = -512
        if trial == 2:
            b[:] = 0xFFFFFFFF
            d[::2] = 511
        got = toeplitz_form_product(d, b)
        exp = O.poly_mul(d.astype(np.int64).astype(np.uint32), b)
        assert np.array_equal(got, exp), trial


def test_core_matrix_walk_reproduces_operand_tiles():
    """Descriptor walk with LBO = SBO = 128 bytes over CM_q (8 x 8 halves)."""
    rng = np.random.default_rng(5)
    N = 1024
    f = hankel_f(rng.integers(0, 2 ** 32, N, dtype=np.uint64).astype(np.uint32))
    fl = np.concatenate([balanced_byte_limbs(f)[0], [0]])
    Q = 2 * N // 8 - 1
    q, r, c = np.meshgrid(np.arange(Q), np.arange(8), np.arange(8), indexing="ij")
    cm = fl[8 * q + r + c].reshape(-1)                   # halves, 64 per core matrix
    # (n0, k0, s): tile origin and K-step; (896, 768, 15) is the last K-step of
    # the last 256-wide chunk of the last coefficient tile: core matrix 254
    for n0, k0, s in ((0, 0, 0), (896, 960, 3), (384, 128, 1), (896, 768, 15)):
        start = (n0 + k0) // 8 * 128 + s * 256            # bytes
        nn = np.arange(128)[:, None]
        kk = np.arange(16)[None, :]
        addr = start + (nn // 8) * 128 + (kk // 8) * 128 + (nn % 8) * 16 + (kk % 8) * 2
        assert addr.max() < cm.size * 2
        tile = cm[addr // 2]
        assert np.array_equal(tile, fl[n0 + nn + k0 + 16 * s + kk])


def test_limbs_recombine_and_stay_bounded():
    x = np.array([0, 1, 127, 128, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 0x807F7F80], np.uint64)
    x = np.concatenate([x, np.random.default_rng(1).integers(0, 2 ** 32, 1000, dtype=np.uint64)])
    limbs = balanced_byte_limbs(x)
    assert all(np.abs(l).max() <= 128 for l in limbs)
    back = sum(limbs[a] << (8 * a) for a in range(4)) & 0xFFFFFFFF
    assert np.array_equal(back, x.astype(np.int64))
    d = np.arange(-512, 512)
    lo, hi = balanced_digit_limbs(d)
    assert np.abs(lo).max() <= 16 and np.abs(hi).max() <= 16
    assert np.array_equal(lo + 32 * hi, d)


def test_worst_case_fp32_accumulation_is_exact():
    """6144 products of magnitude 128 x 16, one sign, summed in fp32 in any
    order: 12,582,912 < 2^24, every partial sum an exact integer."""
    K = 6 * 1024
    a = np.full(K, -128, np.float32)
    b = np.full(K, 16, np.float32)
    acc = np.float32(0)
    for x, y in zip(a, b):
        acc = np.float32(acc + x * y)
    assert int(acc) == -128 * 16 * K == -12582912
    assert abs(int(acc)) < 2 ** 24
    # a random order and blocked (16-term) partial sums, as an MMA would form them
    rng = np.random.default_rng(2)
    p = (a * b)[rng.permutation(K)].reshape(-1, 16)
    blocks = p.sum(axis=1, dtype=np.float32)
    acc = np.float32(0)
    for s in blocks:
        acc = np.float32(acc + s)
    assert int(acc) == -12582912
