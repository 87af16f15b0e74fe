"""32-bit functional units on the GPU engine (the paper's 32-bit variants,
§5: adder, subtractor, shifters, multiplier, divider, flags): decrypted
outputs against the ARMv8 semantics of the oracle's model at width 32 on
random and edge-case operands, one unit's ciphertexts against the oracle's
gate-by-gate evaluation, and the width argument's error cases."""
import numpy as np
import pytest

from gpu_common import ce, ctx, keys, to_dev  # noqa: F401
from oracle import netlists as NL

pytestmark = pytest.mark.gpu
W = 32


def encrypt_operands(ce, sk, a, b, seed, extra=None):
    n = len(a)
    k = 2 * W + (4 if extra is not None else 0)
    out = np.zeros((n, k, 501), np.uint32)
    ctr = 0
    for i in range(n):
        bits = NL.bits(int(a[i]), W) + NL.bits(int(b[i]), W)
        if extra is not None:
            bits += NL.bits(int(extra[i]), 4)
        for j, v in enumerate(bits):
            out[i, j] = ce.ce_encrypt_bit(sk, v, seed, ctr)
            ctr += 1
    return out


def run32(ce, ctx, unit, inp, n_out, cond=0):
    import torch
    c, cid = ctx
    n = inp.shape[0]
    d_out = torch.empty((n, n_out, 501), dtype=torch.int32, device="cuda")
    ce.ce_unit_eval_device_width(c, cid, unit, W, to_dev(inp.view(np.int32)), d_out, n, cond,
                                 torch.cuda.current_stream())
    ce.ce_synchronize(c)
    return d_out.cpu().numpy().view(np.uint32)


def operands(rng, n):
    a = rng.integers(0, 1 << W, n, dtype=np.uint64).astype(np.int64)
    b = rng.integers(0, 1 << W, n, dtype=np.uint64).astype(np.int64)
    a[0], b[0] = 0xFFFFFFFF, 1
    a[1], b[1] = 0x80000000, 31
    a[2], b[2] = 0x7FFFFFFF, 0x80000000
    b[3] = 0
    return a, b


@pytest.mark.parametrize("unit", ["ADD", "SUB", "AND", "ORR", "LSL", "LSR", "ASR", "MUL", "CMP",
                                  "ADD_MUX", "SUB_MUX", "MUL_TREE"])
def test_unit32_semantics(ce, ctx, keys, unit):
    sk, _ = keys
    rng = np.random.default_rng(320 + NL.UNITS.index(unit))
    n = 8
    a, b = operands(rng, n)
    if unit in ("LSL", "LSR", "ASR"):
        b[4:] = rng.integers(0, 64, n - 4)
    out = run32(ce, ctx, unit, encrypt_operands(ce, sk, a, b, 40), 4 if unit == "CMP" else W)
    for i in range(n):
        bits = [ce.ce_decrypt_bit(sk, x) for x in out[i]]
        exp = NL.armv8(unit, int(a[i]), int(b[i]), W)
        got = bits if unit == "CMP" else NL.from_bits(bits)
        assert got == exp, (unit, hex(int(a[i])), hex(int(b[i])), got, exp)


def test_udiv32_semantics(ce, ctx, keys):
    sk, _ = keys
    a = np.array([0xFFFFFFFF, 123456789, 0x80000000], np.int64)
    b = np.array([0x10001, 0, 7], np.int64)
    out = run32(ce, ctx, "UDIV", encrypt_operands(ce, sk, a, b, 41), W)
    for i in range(len(a)):
        got = NL.from_bits([ce.ce_decrypt_bit(sk, x) for x in out[i]])
        assert got == NL.armv8("UDIV", int(a[i]), int(b[i]), W)


def test_csel32_semantics(ce, ctx, keys):
    sk, _ = keys
    rng = np.random.default_rng(33)
    n = 4
    a, b = operands(rng, n)
    f = np.array([0b0010, 0b0000, 0b1001, 0b0110])
    for cond in (0, 10):                                    # EQ, GE
        out = run32(ce, ctx, "CSEL", encrypt_operands(ce, sk, a, b, 42 + cond, f), W, cond)
        for i in range(n):
            got = NL.from_bits([ce.ce_decrypt_bit(sk, x) for x in out[i]])
            assert got == NL.armv8("CSEL", int(a[i]), int(b[i]), W, cond, int(f[i]))


def test_unit32_ciphertexts_match_oracle(ce, ctx, keys, O, full_keys):
    """Every output word of a 32-bit AND equal to the oracle's evaluation of
    its own netlist."""
    sk, _ = keys
    a, b = np.array([0xDEADBEEF], np.int64), np.array([0x0F0F1234], np.int64)
    inp = encrypt_operands(ce, sk, a, b, 43)
    got = run32(ce, ctx, "AND", inp, W)[0]
    exp = NL.eval_ciphertext(full_keys, NL.build("AND", W), list(inp[0]))
    for k in range(W):
        assert (got[k] == exp[k]).all(), k


def test_width_errors(ce, ctx):
    import torch
    c, cid = ctx
    d = torch.zeros((1, 64, 501), dtype=torch.int32, device="cuda")
    for bad in (0, 1, 3, 24, 64):
        with pytest.raises(Exception):
            ce.ce_unit_eval_device_width(c, cid, "ADD", bad, d, d, 1)
