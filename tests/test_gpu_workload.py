"""Full-size checks: the 8192-gate level of 256 16-bit operand pairs (the
adder's first level, 32 gates per pair) in the launch configuration the
benchmark uses; sampled outputs against the oracle, every output against its
truth table, and the output-noise variance against the analytic bound."""
import numpy as np
import pytest

from gpu_common import ce, ctx, keys, encrypt_bits, run_gates_device  # noqa: F401

pytestmark = pytest.mark.gpu

M32 = 2 ** 32


def test_full_level_truth_oracle_and_noise(ce, ctx, keys, O, full_keys):
    sk, _ = keys
    rng = np.random.default_rng(20210103)
    n = 8192
    bits = rng.integers(0, 2, (n, 2))
    ops = np.tile([1, 3], n // 2)              # AND / XOR per bit, as in get_gp
    ca = encrypt_bits(ce, sk, bits[:, 0], 31)
    cb = encrypt_bits(ce, sk, bits[:, 1], 32)
    got = run_gates_device(ce, ctx, ops, ca, cb)
    s = sk.s.astype(np.uint64)
    phase = (got[:, 500].astype(np.uint64) - (got[:, :500].astype(np.uint64) * s).sum(1)) % M32
    phase = np.where(phase >= 2 ** 31, phase.astype(np.int64) - M32, phase.astype(np.int64))
    truth = np.where(ops == 1, bits[:, 0] & bits[:, 1], bits[:, 0] ^ bits[:, 1])
    assert ((phase > 0).astype(int) == truth).all()
    err = (phase - np.where(truth == 1, 2 ** 29, -2 ** 29)) / M32
    p = O.GATE_PARAMS
    var_br = p.n * 2 * p.l * p.N * ((1024 ** 2 - 1) / 12 + 0.25) * p.sigma_bk ** 2
    var_ks = p.N * p.t * 0.75 * p.sigma_lwe ** 2 + p.N / 2 * (2.0 ** -16) ** 2 / 12
    assert err.var() <= 1.1 * (var_br + var_ks), (err.var(), var_br + var_ks)
    idx = np.concatenate([[0, n - 1], rng.choice(n, 14, replace=False)])
    exp = O.gates(full_keys, ops[idx], ca[idx], cb[idx])
    assert (got[idx] == exp).all()
