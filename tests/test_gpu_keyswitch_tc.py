"""Key switching on the tensor cores against the CUDA-core kernel and the oracle.

Both engines compute the fused sample extraction + key switch (§3 "TFHE
Library": one key switch per bootstrapped gate, one per MUX); the tensor-core
engine as a one-hot digit matrix times the key's 11-bit limbs with exact fp32
sums.  Outputs must be bit-identical in all three output modes (packed
gates, MUX pairs, engine descriptors into the arena), with and without the
K split that accumulates partial sums atomically.
"""
import numpy as np
import pytest

from gpu_common import ce, ctx, keys, encrypt_bits, random_ciphertexts, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


def gates_with(ce, c, cid, engine, ops, a, b):
    import torch
    ce.ce_set_keyswitch_config(c, engine)
    n = len(ops)
    out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
    ce.ce_gates_batch_device(c, cid, to_dev(np.asarray(ops, np.uint8)), to_dev(a.view(np.int32)),
                             to_dev(b.view(np.int32)), out, n, torch.cuda.current_stream())
    ce.ce_synchronize(c)
    torch.cuda.synchronize()
    ce.ce_set_keyswitch_config(c, 0)
    return out.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [1, 31, 300, 5000])
def test_gates_tensor_equals_cuda_cores(ce, ctx, n):
    c, cid = ctx
    rng = np.random.default_rng(100 + n)
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    ops = rng.integers(0, 10, n)
    got_tc = gates_with(ce, c, cid, 2, ops, a, b)
    got_cc = gates_with(ce, c, cid, 1, ops, a, b)
    assert (got_tc == got_cc).all()


def test_gates_tensor_matches_oracle(ce, ctx, O, full_keys):
    c, cid = ctx
    rng = np.random.default_rng(7)
    n = 40
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    ops = rng.integers(0, 10, n)
    got = gates_with(ce, c, cid, 2, ops, a, b)
    exp = O.gates(full_keys, ops, a, b)
    assert (got == exp).all()


def test_mux_tensor_equals_cuda_cores(ce, ctx):
    import torch
    c, cid = ctx
    rng = np.random.default_rng(5)
    n = 200
    s, x, y = (random_ciphertexts(rng, n) for _ in range(3))
    res = []
    for engine in (2, 1):
        ce.ce_set_keyswitch_config(c, engine)
        out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
        ce.ce_mux_batch_device(c, cid, to_dev(s.view(np.int32)), to_dev(x.view(np.int32)),
                               to_dev(y.view(np.int32)), out, n, torch.cuda.current_stream())
        ce.ce_synchronize(c)
        torch.cuda.synchronize()
        res.append(out.cpu().numpy())
    ce.ce_set_keyswitch_config(c, 0)
    assert (res[0] == res[1]).all()


@pytest.mark.parametrize("pairs", [3, 64])
def test_unit_tensor_equals_cuda_cores(ce, ctx, keys, pairs):
    import torch
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(pairs)
    bits = rng.integers(0, 2, (pairs, 32))
    ct = encrypt_bits(ce, sk, bits.reshape(-1), 900 + pairs).reshape(pairs, 32, 501)
    d_in = to_dev(ct.view(np.int32))
    res = []
    for engine in (2, 1):
        ce.ce_set_keyswitch_config(c, engine)
        out = torch.empty((pairs, 16, 501), dtype=torch.int32, device="cuda")
        ce.ce_unit_eval_device(c, cid, "ADD", d_in, out, pairs, 0, torch.cuda.current_stream())
        ce.ce_synchronize(c)
        torch.cuda.synchronize()
        res.append(out.cpu().numpy())
    ce.ce_set_keyswitch_config(c, 0)
    assert (res[0] == res[1]).all()
    # and the sums are right
    for i in range(pairs):
        av = sum(int(bits[i, j]) << j for j in range(16))
        bv = sum(int(bits[i, 16 + j]) << j for j in range(16))
        got = sum(ce.ce_decrypt_bit(sk, res[0][i, j].view(np.uint32)) << j for j in range(16))
        assert got == (av + bv) & 0xFFFF


def test_keyswitch_config_rejects_bad_values(ce, ctx):
    c, _ = ctx
    for bad in (-1, 3):
        with pytest.raises(Exception):
            ce.ce_set_keyswitch_config(c, bad)
