"""GPU path vs the plain CPU oracle: every ciphertext word must be equal
(bit-exact; all arithmetic on both sides is exact integer arithmetic)."""
import numpy as np
import pytest

from gpu_common import (ce, ctx, keys, encrypt_bits, random_ciphertexts,  # noqa: F401
                        run_gates_device, to_dev)

pytestmark = pytest.mark.gpu


def test_negacyclic_mul_matches_oracle(ce, ctx, O):
    import torch
    c, _ = ctx
    rng = np.random.default_rng(11)
    n = 37  # odd: the last block carries one product
    d = rng.integers(-512, 512, (n, 1024)).astype(np.int16)
    d[3] = rng.integers(-2 ** 13, 2 ** 13 + 1, 1024)      # full documented range
    d[4] = -2 ** 13
    d[6] = 2 ** 13
    k = rng.integers(0, 2 ** 32, (n, 1024), dtype=np.uint64).astype(np.uint32)
    k[5] = 0xFFFFFFFF
    k[4] = 0x80000000      # every term +2^44: the exact sum is 2^54, the bound
    k[6] = 0x80000000      # every term -2^44: -2^54
    out = torch.empty((n, 1024), dtype=torch.int32, device="cuda")
    ce.ce_negacyclic_mul_device(c, to_dev(d), to_dev(k.view(np.int32)), out, n)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n):
        exp = O.poly_mul(d[i].astype(np.int64).astype(np.uint32), k[i])
        assert (got[i] == exp).all(), i


def test_truth_tables_bit_exact(ce, ctx, keys, O, full_keys):
    sk, _ = keys
    ops, bits = [], []
    for op in ("NAND", "AND", "OR", "XOR"):
        for a in (0, 1):
            for b in (0, 1):
                ops.append(O.GATE_ID[op])
                bits.append((a, b))
    bits = np.array(bits)
    ca = encrypt_bits(ce, sk, bits[:, 0], 5)
    cb = encrypt_bits(ce, sk, bits[:, 1], 6)
    got = run_gates_device(ce, ctx, ops, ca, cb)
    exp = O.gates(full_keys, ops, ca, cb)
    for i, op in enumerate(ops):
        assert ce.ce_decrypt_bit(sk, got[i]) == O.TRUTH[O.GATES[op]](*bits[i])
        assert (got[i] == exp[i]).all(), (O.GATES[op], bits[i])


def test_all_gates_random_inputs_bit_exact(ce, ctx, O, full_keys):
    rng = np.random.default_rng(12)
    ops = list(range(10)) * 2
    a, b = random_ciphertexts(rng, 20), random_ciphertexts(rng, 20)
    got = run_gates_device(ce, ctx, ops, a, b)
    assert (got == O.gates(full_keys, ops, a, b)).all()


def test_skip_path_and_trivial_inputs(ce, ctx, O, full_keys):
    """Inputs whose modulus switch gives abar_i = 0 for many i (the CMux step
    is the identity) and trivial ciphertexts (a = 0)."""
    rng = np.random.default_rng(13)
    a, b = random_ciphertexts(rng, 6), random_ciphertexts(rng, 6)
    a[0, :500] = 0
    b[0, :500] = 0
    a[1, ::2] = 0x000FFFFF          # rounds to 0
    b[1, ::3] = 0xFFF00000          # rounds to 2048 = 0
    a[2, :500] = 0                  # trivial CONSTANT-like inputs
    b[2, :500] = 0
    a[2, 500], b[2, 500] = 0x20000000, 0xE0000000
    ops = [0, 1, 2, 3, 4, 5]
    got = run_gates_device(ce, ctx, ops, a, b)
    assert (got == O.gates(full_keys, ops, a, b)).all()


@pytest.mark.parametrize("gpb", [1, 2, 3, 4])
def test_launch_shapes_agree_and_match_oracle(ce, ctx, O, full_keys, gpb):
    """Several blocks, several gate groups per block and a ragged tail, for
    each gates-per-block variant; sampled outputs checked against the oracle,
    all outputs against each other."""
    c, cid = ctx
    rng = np.random.default_rng(100 + gpb)
    n = 1201
    ops = rng.integers(0, 10, n)
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    ce.ce_set_blind_rotate_config(c, gpb, 0)
    try:
        got = run_gates_device(ce, ctx, ops, a, b)
    finally:
        ce.ce_set_blind_rotate_config(c, 0, 0)
    ref = run_gates_device(ce, ctx, ops, a, b)   # autotuned shape
    assert (got == ref).all()
    idx = np.unique(np.concatenate([rng.choice(n, 6, replace=False), [0, n - 1]]))
    exp = O.gates(full_keys, ops[idx], a[idx], b[idx])
    assert (got[idx] == exp).all()


@pytest.mark.parametrize("gpb,n", [(4, 708), (4, 808), (2, 404)])
def test_part_filled_last_round_runs_in_a_smaller_shape(ce, ctx, O, full_keys, gpb, n):
    """A batch whose gate groups leave the last round over the SMs part
    filled runs its whole rounds in the chosen shape and the remaining gates
    in a shape with fewer gates per block (one gate per block for up to one
    gate per SM, two for up to two): outputs equal the one-gate-per-block
    shape's everywhere and the oracle on sampled gates of both parts."""
    import torch
    c, cid = ctx
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    rng = np.random.default_rng(300 + n)
    ops = rng.integers(0, 10, n)
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    counts = {}
    for shape in (gpb, 1):
        ce.ce_set_blind_rotate_config(c, shape, 0)
        try:
            out = run_gates_device(ce, ctx, ops, a, b)
            counts[shape] = ce.ce_last_launch_count(c)
        finally:
            ce.ce_set_blind_rotate_config(c, 0, 0)
        if shape == gpb:
            got = out
    assert (got == out).all()
    groups = -(-n // gpb)
    whole = (groups // sms) * sms * gpb
    tail = n - whole
    split = groups > sms and groups % sms != 0 and (tail <= sms or (gpb == 4 and tail <= 2 * sms))
    assert counts[gpb] == counts[1] + (1 if split else 0)
    idx = np.unique(np.concatenate([rng.choice(n, 4, replace=False),
                                    [0, max(whole - 1, 0), min(whole, n - 1), n - 1]]))
    exp = O.gates(full_keys, ops[idx], a[idx], b[idx])
    assert (got[idx] == exp).all()


def test_host_buffer_api_matches_device_api(ce, ctx, keys, O):
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(14)
    n = 40
    bits = rng.integers(0, 2, (n, 2))
    ca, cb = encrypt_bits(ce, sk, bits[:, 0], 7), encrypt_bits(ce, sk, bits[:, 1], 8)
    ops = rng.integers(0, 10, n).astype(np.uint8)
    host = ce.ce_gates_batch(c, cid, ops, ca, cb)
    dev = run_gates_device(ce, ctx, ops, ca, cb)
    assert (host == dev).all()
    one = ce.ce_gate(c, cid, int(ops[3]), ca[3], cb[3])
    assert (one == dev[3]).all()
    for i in range(n):
        assert ce.ce_decrypt_bit(sk, host[i]) == O.TRUTH[O.GATES[ops[i]]](*bits[i])


def test_mux_bit_exact(ce, ctx, keys, O, full_keys):
    import torch
    c, cid = ctx
    sk, _ = keys
    sel = np.array([(i >> 2) & 1 for i in range(8)] + [1, 0])
    x = np.array([(i >> 1) & 1 for i in range(8)] + [0, 1])
    y = np.array([i & 1 for i in range(8)] + [1, 1])
    ca, cb, cc = (encrypt_bits(ce, sk, v, s) for v, s in ((sel, 21), (x, 22), (y, 23)))
    n = len(sel)
    out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
    ce.ce_mux_batch_device(c, cid, to_dev(ca.view(np.int32)), to_dev(cb.view(np.int32)),
                           to_dev(cc.view(np.int32)), out, n)
    ce.ce_synchronize(c)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n):
        assert ce.ce_decrypt_bit(sk, got[i]) == (x[i] if sel[i] else y[i])
        if i < 4:
            assert (got[i] == O.mux(full_keys, ca[i], cb[i], cc[i])).all()


def test_empty_batch_and_errors(ce, ctx):
    import torch
    c, cid = ctx
    z = torch.empty((0, 501), dtype=torch.int32, device="cuda")
    ce.ce_gates_batch_device(c, cid, torch.empty(0, dtype=torch.uint8, device="cuda"), z, z, z, 0)
    assert ce.ce_last_launch_count(c) == 0
    one = torch.zeros((1, 501), dtype=torch.int32, device="cuda")
    ops = torch.zeros(1, dtype=torch.uint8, device="cuda")
    with pytest.raises(ce.CeError) as ei:
        ce.ce_gates_batch_device(c, cid + 77, ops, one, one, one, 1)
    assert ei.value.code == -6
    with pytest.raises(ce.CeError) as ei:      # null device buffer
        ce.ce_gates_batch_device(c, cid, ops, 0, one, one, 1)
    assert ei.value.code == -1
    bad = torch.full((1,), 200, dtype=torch.uint8, device="cuda")   # not a gate opcode
    ce.ce_gates_batch_device(c, cid, bad, one, one, one, 1)
    with pytest.raises(ce.CeError) as ei:
        ce.ce_synchronize(c)
    assert ei.value.code == -1
    ce.ce_synchronize(c)                        # the flag was consumed
    with pytest.raises(ce.CeError):
        ce.ce_set_blind_rotate_config(c, 5, 0)      # no such launch shape


def test_autotuner_installs_shapes_and_keeps_results(ce, ctx, O, full_keys):
    import numpy as np
    from gpu_common import random_ciphertexts, run_gates_device
    c, cid = ctx
    rng = np.random.default_rng(55)
    ops = rng.integers(0, 10, 40)
    a, b = random_ciphertexts(rng, 40), random_ciphertexts(rng, 40)
    before = run_gates_device(ce, ctx, ops, a, b)
    table = ce.ce_autotune(c, cid)
    assert set(table.values()) <= {1, 2, 3, 4} and min(table) == 1 and max(table) >= 9728
    after = run_gates_device(ce, ctx, ops, a, b)
    assert (before == after).all()
