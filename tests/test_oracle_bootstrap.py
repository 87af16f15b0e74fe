"""Pins of the oracle's keys, encryption, blind rotation, sample extraction,
key switching and gates against closed forms, exact identities, truth tables
and the noise bound."""
import math

import numpy as np
import pytest

from conftest import signed32

M32 = 1 << 32


def trlwe_phase(O, acc, K):
    """B - A*K using the oracle product (itself pinned by brute force)."""
    return (acc[1].astype(np.uint64) - O.poly_mul(acc[0], K)) % M32


def rotate_const(N, mu, k):
    """X^k * (mu * sum_j X^j) written out coefficient by coefficient."""
    k %= 2 * N
    out = []
    for j in range(N):
        # coefficient j of X^k v: v_{j-k} (+) if j >= k else -v_{j-k+N}, X^N = -1
        if k < N:
            v = mu if j >= k else -mu
        else:
            v = -mu if j >= k - N else mu
        out.append(v % M32)
    return np.array(out, dtype=np.uint64)


def test_bsk_rows_encrypt_gadget_times_key_bit(O, tiny_keys):
    p, k = tiny_keys.params, tiny_keys
    for i in range(p.n):
        for r in range(2 * p.l):
            c, pp = divmod(r, p.l)
            h = 1 << (32 - p.Bgbit * (pp + 1))
            row = k.bsk[i, r]
            ph = trlwe_phase(O, row, k.K).astype(np.int64)
            if c == 1:
                ph[0] -= int(k.s[i]) * h
            else:  # (a + s h, a K + e): phase = e - s h K
                ph = (ph + int(k.s[i]) * h * k.K.astype(np.int64)) % M32
            e = signed32(ph)
            assert np.abs(e).max() <= 8 * p.sigma_bk * M32 + 1


def test_ksk_rows_encrypt_digit_times_key(O, tiny_keys):
    p, k = tiny_keys.params, tiny_keys
    for j in range(p.N):
        for q in range(p.t):
            for v in range(1 << p.basebit):
                ph = O.phase(p, k.s, k.ksk[j, q, v])
                msg = (v * int(k.K[j]) << (32 - p.basebit * (q + 1))) % M32
                assert abs(int(signed32(ph - msg))) <= 8 * p.sigma_lwe * M32


def test_encrypt_decrypt_and_noise(O, full_keys):
    p = full_keys.params
    errs = []
    for i in range(400):
        bit = i & 1
        c = O.encrypt(p, full_keys.s, bit, 31, i)
        assert O.decrypt(p, full_keys.s, c) == bit
        errs.append(int(signed32(O.phase(p, full_keys.s, c) - (O.MU if bit else -O.MU))))
    e = np.array(errs) / M32
    assert abs(e.std() / p.sigma_lwe - 1) < 5 * math.sqrt(0.5 / len(e))


def modswitched(O, p, c):
    return [O.modswitch(int(x), p.N) for x in c[:p.n]], O.modswitch(int(c[p.n]), p.N)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_blind_rotation_closed_form_noise_free(O, seed):
    """With a noise-free bootstrapping key, Dec_K(ACC) rounded to multiples of
    mu equals X^(-phi) v exactly, phi = bbar - sum abar_i s_i mod 2N."""
    p = O.Params(n=40, N=128, sigma_bk=0.0)
    keys = O.keygen(p, 1000 + seed)
    rng = np.random.default_rng(seed)
    abar = rng.integers(0, 2 * p.N, p.n).astype(np.uint32)
    abar[::7] = 0
    bbar = int(rng.integers(0, 2 * p.N))
    acc = O.blind_rotate(p, keys.bsk, abar, bbar)
    ph = trlwe_phase(O, acc, keys.K)
    phi = (bbar - int((abar.astype(np.int64) * keys.s).sum())) % (2 * p.N)
    expected = rotate_const(p.N, O.MU, -phi)
    err = signed32(ph - expected)
    # decomposition rounding only: |err| <= 2 * N * n (here far below mu/2)
    assert np.abs(err).max() <= 2 * p.N * p.n
    got = np.round(signed32(ph) / O.MU).astype(np.int64) * O.MU % M32
    assert (got == expected).all()


def test_blind_rotation_closed_form_full_size(O):
    p = O.Params(sigma_bk=0.0)
    keys = O.keygen(p, 4242)
    rng = np.random.default_rng(4)
    abar = rng.integers(0, 2 * p.N, p.n).astype(np.uint32)
    bbar = int(rng.integers(0, 2 * p.N))
    acc = O.blind_rotate(p, keys.bsk, abar, bbar)
    ph = trlwe_phase(O, acc, keys.K)
    phi = (bbar - int((abar.astype(np.int64) * keys.s).sum())) % (2 * p.N)
    err = signed32(ph - rotate_const(p.N, O.MU, -phi))
    assert np.abs(err).max() <= 2 * p.N * p.n


def test_sample_extract_identity(O, tiny_keys):
    p = tiny_keys.params
    rng = np.random.default_rng(8)
    for _ in range(10):
        acc = rng.integers(0, M32, (2, p.N), dtype=np.uint64).astype(np.uint32)
        big = O.sample_extract(p, acc)
        # phase of the extracted LWE under K equals coefficient 0 of the TRLWE phase
        lwe_phase = (int(big[p.N]) - int((big[:p.N].astype(np.uint64) * tiny_keys.K).sum())) % M32
        assert lwe_phase == int(trlwe_phase(O, acc, tiny_keys.K)[0])


def test_key_switch_exact_when_noise_free_and_rounded(O):
    p = O.Params(n=30, N=64, sigma_lwe=0.0)
    keys = O.keygen(p, 55)
    rng = np.random.default_rng(2)
    for trial in range(20):
        big = rng.integers(0, M32, p.N + 1, dtype=np.uint64).astype(np.uint32)
        if trial % 2 == 0:  # a'_j already on the 16-bit grid: switch is exact
            big[:p.N] &= np.uint32(0xFFFF0000)
        out = O.key_switch(p, keys.ksk, big)
        before = (int(big[p.N]) - int((big[:p.N].astype(np.uint64) * keys.K).sum())) % M32
        diff = int(signed32(O.phase(p, keys.s, out) - before))
        if trial % 2 == 0:
            assert diff == 0
        else:
            assert abs(diff) <= p.N * (1 << 15)


def truth_table_check(O, keys, ops, pairs, seed):
    p = keys.params
    c1 = [O.encrypt(p, keys.s, a, seed, 2 * i) for i, (a, b) in enumerate(pairs)]
    c2 = [O.encrypt(p, keys.s, b, seed, 2 * i + 1) for i, (a, b) in enumerate(pairs)]
    out = O.gates(keys, ops, np.stack(c1), np.stack(c2))
    for i, (op, (a, b)) in enumerate(zip(ops, pairs)):
        assert O.decrypt(p, keys.s, out[i]) == O.TRUTH[op](a, b), (op, a, b)


def test_gate_truth_tables_small(O, tiny_keys):
    ops, pairs = [], []
    for op in O.GATES:
        for a in (0, 1):
            for b in (0, 1):
                ops.append(op)
                pairs.append((a, b))
    truth_table_check(O, tiny_keys, ops, pairs, 9)


def test_mux_small(O, tiny_keys):
    p = tiny_keys.params
    for i in range(8):
        a, b, c = (i >> 2) & 1, (i >> 1) & 1, i & 1
        ca, cb, cc = (O.encrypt(p, tiny_keys.s, v, 3, 3 * i + j) for j, v in enumerate((a, b, c)))
        assert O.decrypt(p, tiny_keys.s, O.mux(tiny_keys, ca, cb, cc)) == (b if a else c)


def test_not_and_constant(O, tiny_keys):
    p = tiny_keys.params
    for bit in (0, 1):
        assert O.decrypt(p, tiny_keys.s, O.constant(p, bit)) == bit
        c = O.encrypt(p, tiny_keys.s, bit, 4, bit)
        assert O.decrypt(p, tiny_keys.s, O.not_(p, c)) == 1 - bit


@pytest.mark.slow
def test_gate_truth_tables_full_size(O, full_keys):
    """Every gate once plus NAND/AND/OR/XOR on all four input pairs."""
    ops, pairs = [], []
    for i, op in enumerate(O.GATES):
        ops.append(op)
        pairs.append(((i >> 1) & 1, i & 1))
    for op in ("NAND", "AND", "OR", "XOR"):
        for a in (0, 1):
            for b in (0, 1):
                ops.append(op)
                pairs.append((a, b))
    truth_table_check(O, full_keys, ops, pairs, 21)


def test_output_noise_within_bound(O):
    """Empirical output-noise variance of bootstrapped gates against the
    analytic bound: n * 2l * N * E[d^2] * sigma_bk^2 (external products)
    + N * t * (1 - 2^-basebit) * sigma_ks^2 (key switch) + rounding terms."""
    p = O.Params(n=50, N=128, sigma_bk=2.0 ** -22, sigma_lwe=2.0 ** -17)
    keys = O.keygen(p, 606)
    count = 1536
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, (count, 2))
    c1 = np.stack([O.encrypt(p, keys.s, int(b), 8, 2 * i) for i, b in enumerate(bits[:, 0])])
    c2 = np.stack([O.encrypt(p, keys.s, int(b), 8, 2 * i + 1) for i, b in enumerate(bits[:, 1])])
    out = O.gates(keys, ["NAND"] * count, c1, c2)
    expect = np.where(1 - (bits[:, 0] & bits[:, 1]) == 1, O.MU, -O.MU)
    err = np.array([int(signed32(O.phase(p, keys.s, o) - e)) for o, e in zip(out, expect)]) / M32
    Bg = 1 << p.Bgbit
    ed2 = (Bg * Bg - 1) / 12.0 + 0.25
    var_br = p.n * 2 * p.l * p.N * ed2 * p.sigma_bk ** 2
    var_ks = p.N * p.t * (1 - 2.0 ** -p.basebit) * p.sigma_lwe ** 2
    var_round = p.N / 2 * (2.0 ** -(p.t * p.basebit)) ** 2 / 12   # key-switch rounding
    bound = var_br + var_ks + var_round
    var = err.var()
    assert var <= 1.15 * bound, (var, bound)
    assert var >= 0.5 * bound, (var, bound)   # the noise terms are really there


def test_gate_lincomb_maximum_margin(O):
    """With bits encoded as +-1/8, the linear part of each gate must put every
    input row on its truth-table side of the decision boundaries {0, 1/2} with
    the largest margin the encoding allows: 1/8 for the one-weight gates and
    1/4 for XOR/XNOR (weights 2).  This fixes the gate constant uniquely."""
    p = O.Params(n=4, N=64)
    for op in O.GATES:
        margins = []
        for a in (0, 1):
            for b in (0, 1):
                lin = O.gate_lincomb(p, op, O.constant(p, a), O.constant(p, b))
                assert (lin[:p.n] == 0).all()
                ph = int(lin[p.n]) / M32            # phase in [0, 1)
                truth = O.TRUTH[op](a, b)
                assert (0 < ph < 0.5) == bool(truth), (op, a, b, ph)
                margins.append(min(ph % 0.5, 0.5 - ph % 0.5))
        best = 0.25 if op in ("XOR", "XNOR") else 0.125
        assert min(margins) == best, (op, margins)
