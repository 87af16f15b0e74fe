"""Functional units on the GPU engine: decrypted outputs vs ARMv8 semantics
over many operand sets; whole-unit ciphertexts vs the oracle's gate-by-gate
evaluation of its own netlist (bit-exact); graph replay vs eager launches."""
import numpy as np
import pytest

from gpu_common import ce, ctx, keys, to_dev  # noqa: F401
from oracle import netlists as NL

pytestmark = pytest.mark.gpu
W = 16


def enc_operands(ce, sk, vals, seed):
    """[n][len(vals[0])*...]: bit-sliced encryptions, input order a bits, b bits (, flags)."""
    n, k = vals.shape
    out = np.zeros((n, k, 501), np.uint32)
    ctr = 0
    for i in range(n):
        for j in range(k):
            out[i, j] = ce.ce_encrypt_bit(sk, int(vals[i, j]), seed, ctr)
            ctr += 1
    return out


def operand_bits(a, b, extra=None):
    cols = [(a >> i) & 1 for i in range(W)] + [(b >> i) & 1 for i in range(W)]
    if extra is not None:
        cols += [(extra >> i) & 1 for i in range(4)]
    return np.stack(cols, axis=1)


def run_unit(ce, ctx, unit, inp, n_out, cond=0):
    import torch
    c, cid = ctx
    n = inp.shape[0]
    d_in = to_dev(inp.view(np.int32))
    d_out = torch.empty((n, n_out, 501), dtype=torch.int32, device="cuda")
    ce.ce_unit_eval_device(c, cid, unit, d_in, d_out, n, cond, torch.cuda.current_stream())
    ce.ce_synchronize(c)
    return d_out.cpu().numpy().view(np.uint32)


def decrypt_all(ce, sk, out):
    return np.array([[ce.ce_decrypt_bit(sk, x) for x in row] for row in out])


def operands(rng, n):
    a = rng.integers(0, 1 << W, n)
    b = rng.integers(0, 1 << W, n)
    a[0], b[0] = 0xFFFF, 1
    a[1], b[1] = 1234, 1234
    a[2], b[2] = 0x8000, 0x7FFF
    b[3] = 0
    return a, b


@pytest.mark.parametrize("unit", ["ADD", "ADD_RIPPLE", "SUB", "AND", "ORR", "LSL", "MUL", "CMP",
                                  "LSR", "ASR", "EOR", "ORN", "ADDS", "SUBS", "SMULL", "UMULL",
                                  "ADD_MUX", "SUB_MUX", "MUL_TREE"])
def test_unit_semantics(ce, ctx, keys, unit):
    sk, _ = keys
    rng = np.random.default_rng(sum(map(ord, unit)))
    n = 40
    a, b = operands(rng, n)
    n_out = {"CMP": 4, "ADDS": W + 4, "SUBS": W + 4, "SMULL": 2 * W, "UMULL": 2 * W}.get(unit, W)
    out = run_unit(ce, ctx, unit, enc_operands(ce, sk, operand_bits(a, b), 5), n_out)
    bits = decrypt_all(ce, sk, out)
    for i in range(n):
        exp = NL.armv8(unit, int(a[i]), int(b[i]), W)
        if unit == "CMP":
            got = list(bits[i])
        elif unit in ("ADDS", "SUBS"):
            got = [NL.from_bits(bits[i][:W])] + list(bits[i][W:])
        else:
            got = NL.from_bits(bits[i])
        assert got == exp, (unit, int(a[i]), int(b[i]), got, exp)


@pytest.mark.parametrize("unit", ["UDIV", "UDIV_MUX"])
def test_udiv_semantics(ce, ctx, keys, unit):
    sk, _ = keys
    rng = np.random.default_rng(9)
    n = 12
    a, b = operands(rng, n)
    b[4] = 1
    b[5] = rng.integers(1, 16)
    out = run_unit(ce, ctx, unit, enc_operands(ce, sk, operand_bits(a, b), 6), W)
    bits = decrypt_all(ce, sk, out)
    for i in range(n):
        assert NL.from_bits(bits[i]) == NL.armv8(unit, int(a[i]), int(b[i]), W)


@pytest.mark.parametrize("cond", [0, 8, 10, 12])
def test_csel_semantics(ce, ctx, keys, cond):
    sk, _ = keys
    rng = np.random.default_rng(cond)
    n = 16
    a, b = operands(rng, n)
    f = np.arange(n) % 16
    out = run_unit(ce, ctx, "CSEL", enc_operands(ce, sk, operand_bits(a, b, f), 7), W, cond)
    bits = decrypt_all(ce, sk, out)
    for i in range(n):
        assert NL.from_bits(bits[i]) == NL.armv8("CSEL", int(a[i]), int(b[i]), W, cond, int(f[i]))


def test_graph_replay_equals_eager(ce, ctx, keys):
    c, _ = ctx
    sk, _ = keys
    rng = np.random.default_rng(3)
    a, b = operands(rng, 24)
    inp = enc_operands(ce, sk, operand_bits(a, b), 8)
    g1 = run_unit(ce, ctx, "ADD", inp, W)
    g2 = run_unit(ce, ctx, "ADD", inp, W)            # replay of the captured graph
    ce.ce_set_unit_graphs(c, False)
    try:
        eager = run_unit(ce, ctx, "ADD", inp, W)
    finally:
        ce.ce_set_unit_graphs(c, True)
    assert (g1 == g2).all() and (g1 == eager).all()


@pytest.mark.parametrize("unit,cond", [("ADD", 0), ("CSEL", 12)])
def test_one_launch_per_gate_equals_level_batching(ce, ctx, keys, unit, cond):
    """With level batching off every gate runs as launches of its own (its
    linear combination and one-gate blind rotation per bootstrap, its
    extraction + key switch per gate output): the same ciphertexts as the
    level-batched engine, MUX gates (CSEL) included, and exactly that many
    launches plus the operand copies."""
    c, _ = ctx
    sk, _ = keys
    rng = np.random.default_rng(31)
    a, b = rng.integers(0, 1 << W, 2), rng.integers(0, 1 << W, 2)
    f = np.array([4, 9]) if unit == "CSEL" else None   # NZCV bits N|Z<<1|C<<2|V<<3
    inp = enc_operands(ce, sk, operand_bits(a, b, f), 12)
    ce.ce_set_unit_graphs(c, False)
    try:
        batched = run_unit(ce, ctx, unit, inp, W, cond)
        batched_launches = ce.ce_last_launch_count(c)
        ce.ce_set_level_batching(c, False)
        try:
            per_gate = run_unit(ce, ctx, unit, inp, W, cond)
            per_gate_launches = ce.ce_last_launch_count(c)
        finally:
            ce.ce_set_level_batching(c, True)
    finally:
        ce.ce_set_unit_graphs(c, True)
    assert (per_gate == batched).all()
    info = ce.ce_unit_info(unit, cond=cond)   # two instances: jobs = bootstraps, outputs = gates
    assert per_gate_launches == 2 + 2 * (2 * info["n_bootstraps"]) + 2 * info["n_gates"]
    assert per_gate_launches > 10 * batched_launches


@pytest.mark.parametrize("unit", ["AND", "LSL", "ADD", "ASR", "ADD_MUX", "SUB_MUX"])
def test_unit_ciphertexts_match_oracle(ce, ctx, keys, O, full_keys, unit):
    """One instance, every output word equal to the oracle evaluating its own
    (independently built) netlist gate by gate."""
    sk, _ = keys
    a, b = np.array([0xBEEF]), np.array([5 if unit in ("LSL", "ASR") else 0x0137])
    inp = enc_operands(ce, sk, operand_bits(a, b), 11)
    got = run_unit(ce, ctx, unit, inp, W)[0]
    net = NL.build(unit, W)
    exp = NL.eval_ciphertext(full_keys, net, list(inp[0]))
    for k in range(W):
        assert (got[k] == exp[k]).all(), (unit, k)
    assert NL.from_bits(decrypt_all(ce, sk, got[None])[0]) == NL.armv8(unit, 0xBEEF, int(b[0]), W)


def test_graph_replay_after_scratch_growth(ce, ctx, keys):
    """A captured unit graph must not keep using scratch that a larger later
    call replaced: replay after growth equals a fresh eager evaluation."""
    import torch
    from gpu_common import random_ciphertexts, run_gates_device
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(31)
    a, b = operands(rng, 8)
    inp = enc_operands(ce, sk, operand_bits(a, b), 12)
    d_in = to_dev(inp.view(np.int32))
    d_out = torch.empty((8, W, 501), dtype=torch.int32, device="cuda")
    ce.ce_unit_eval_device(c, cid, "ORR", d_in, d_out, 8, 0)      # captures the graph
    ce.ce_synchronize(c)
    first = d_out.clone()
    n = 20000                                                       # grows the scratch
    ops = rng.integers(0, 10, n)
    run_gates_device(ce, ctx, ops, random_ciphertexts(rng, n), random_ciphertexts(rng, n))
    d_out.zero_()
    ce.ce_unit_eval_device(c, cid, "ORR", d_in, d_out, 8, 0)      # same buffers: replay
    ce.ce_synchronize(c)
    assert torch.equal(first, d_out)
    bits = decrypt_all(ce, sk, d_out.cpu().numpy().view(np.uint32))
    for i in range(8):
        assert NL.from_bits(bits[i]) == int(a[i]) | int(b[i])


def test_host_buffer_unit_call_equals_device_call(ce, ctx, keys):
    """ce_unit_eval (host buffers in and out) returns exactly what
    ce_unit_eval_device returns on the same inputs, at 16 and 32 bits."""
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(41)
    a, b = operands(rng, 6)
    inp = enc_operands(ce, sk, operand_bits(a, b), 13)
    dev = run_unit(ce, ctx, "SUB", inp, W)
    host = ce.ce_unit_eval(c, cid, "SUB", inp)
    assert host.shape == dev.shape and (host == dev).all()
    assert ce.ce_last_launch_count(c) > 0
    bits = decrypt_all(ce, sk, host)
    for i in range(6):
        assert NL.from_bits(bits[i]) == (int(a[i]) - int(b[i])) & 0xFFFF
    # width 32, AND: one level
    w32 = np.stack([np.stack([ce.ce_encrypt_bit(sk, int(x), 14, 64 * i + j)
                              for j, x in enumerate(rng.integers(0, 2, 64))]) for i in range(3)])
    got = ce.ce_unit_eval(c, cid, "AND", w32, width=32)
    import torch
    d_out = torch.empty((3, 32, 501), dtype=torch.int32, device="cuda")
    ce.ce_unit_eval_device_width(c, cid, "AND", 32, to_dev(w32.view(np.int32)), d_out, 3)
    ce.ce_synchronize(c)
    assert (got == d_out.cpu().numpy().view(np.uint32)).all()
