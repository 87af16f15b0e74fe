"""Ciphertext parity inside whole functional units, programs and a serving
mix: the engine records sampled gates of every level exactly as the GPU
evaluated them (ce_trace_enable), and the plain CPU oracle recomputes each
from the GPU's own inputs; all 501 words must agree.  This covers the
16-bit array multiplier (§5 "Multiplier") in both external-product forms, a
register program through CMP, CSEL and the barrel shifter (§5 "Shifter",
§6 "Conditional Flags"), and one request inside a four-client serving mix
(§4 "Cloud service model"), each at every level."""
import numpy as np
import pytest

from gpu_common import MASTER_SEED, ce, ctx, keys, to_dev  # noqa: F401
from oracle import netlists as NL

pytestmark = pytest.mark.gpu
W = 16


def enc_word(ce, sk, v, seed, base):
    return np.stack([ce.ce_encrypt_bit(sk, (v >> j) & 1, seed, base + j) for j in range(W)])


def dec_word(ce, sk, bits):
    return sum(ce.ce_decrypt_bit(sk, bits[j]) << j for j in range(W))


def oracle_check(O, keys_by_client, recs):
    """Recompute every traced gate with the oracle; returns the mismatches."""
    p = None
    bad = []
    for client, okeys in keys_by_client.items():
        p = okeys.params
        mine = recs[recs["client"] == client]

        def inp(r, i):
            x = r["inp"][i]
            return O.not_(p, x) if r["neg"][i] else x

        plain = mine[mine["op"] < 10]
        if len(plain):
            exp = O.gates(okeys, plain["op"], [inp(r, 0) for r in plain],
                          [inp(r, 1) for r in plain])
            bad += [(int(r["tick"]), int(r["index"])) for r, e in zip(plain, exp)
                    if not (r["out"] == e).all()]
        mux = mine[mine["op"] == 10]
        if len(mux):
            exp = O.muxes(okeys, [inp(r, 0) for r in mux], [inp(r, 1) for r in mux],
                          [inp(r, 2) for r in mux])
            bad += [(int(r["tick"]), int(r["index"])) for r, e in zip(mux, exp)
                    if not (r["out"] == e).all()]
    return bad


@pytest.mark.parametrize("form,per_level", [(0, 6), (1, 3)])
def test_mul_levels_match_oracle(ce, ctx, keys, O, full_keys, form, per_level):
    """16-bit MUL (557 bootstraps, 30 levels) on two operand pairs: sampled
    gates of every level, MUX full-adder carries included, against the
    oracle on the GPU's level inputs; transform form (0) and Toeplitz
    tensor-core form (1) of the external products."""
    import torch
    c, cid = ctx
    sk, _ = keys
    a, b = np.array([0xBEEF, 0x1234]), np.array([0x7A31, 0xFFFF])
    bits = np.stack([[(int(a[i]) >> j) & 1 for j in range(W)] + [(int(b[i]) >> j) & 1
                                                                   for j in range(W)]
                     for i in range(2)])
    inp = np.stack([np.stack([ce.ce_encrypt_bit(sk, int(x), 40 + form, 32 * i + j)
                              for j, x in enumerate(bits[i])]) for i in range(2)])
    d_in = to_dev(inp.view(np.int32))
    d_out = torch.empty((2, W, 501), dtype=torch.int32, device="cuda")
    ce.ce_set_external_product_form(c, form)
    try:
        ce.ce_trace_enable(c, per_level, 4096)
        ce.ce_unit_eval_device(c, cid, "MUL", d_in, d_out, 2, 0)
        ce.ce_synchronize(c)
        recs, seen = ce.ce_trace_read(c)
    finally:
        ce.ce_trace_enable(c, 0)
        ce.ce_set_external_product_form(c, 0)
    depth = ce.ce_unit_info("MUL")["depth"]
    assert seen == len(recs) > 0
    assert sorted(set(recs["tick"].tolist())) == list(range(depth)), "a level was not sampled"
    assert (recs["op"] == 10).any(), "no MUX (full-adder carry) was sampled"
    assert (recs["client"] == cid).all()
    assert oracle_check(O, {cid: full_keys}, recs) == []
    out = d_out.cpu().numpy().view(np.uint32)
    for i in range(2):
        assert dec_word(ce, sk, out[i]) == (int(a[i]) * int(b[i])) & 0xFFFF


def test_program_levels_match_oracle(ce, ctx, keys, O, full_keys):
    """A register program through ADD, CMP, CSEL (GT), the LSL barrel and
    SUB: sampled gates of every tick against the oracle; final registers
    against the plaintext machine."""
    c, cid = ctx
    sk, _ = keys
    vals = [0x9C41, 0x0005]
    for r, v in enumerate(vals):
        ce.ce_reg_write(c, cid, r, enc_word(ce, sk, v, 50, 16 * r))
    prog = [("ADD", 2, 0, 1), ("CMP", 0, 0, 1), ("CSEL", 3, 2, 0, 0, 12), ("LSL", 4, 3, 1),
            ("SUB", 5, 4, 0)]
    ce.ce_trace_enable(c, 4, 4096)
    try:
        ce.ce_exec(c, cid, [ce.insn(*x) for x in prog])
        recs, seen = ce.ce_trace_read(c)
    finally:
        ce.ce_trace_enable(c, 0)
    ticks = sum(ce.ce_unit_info(u, cond=12 if u == "CSEL" else 0)["depth"]
                for u in ("ADD", "CMP", "CSEL", "LSL", "SUB"))
    assert seen == len(recs)
    assert sorted(set(recs["tick"].tolist())) == list(range(ticks))
    assert oracle_check(O, {cid: full_keys}, recs) == []
    # plaintext machine
    reg, nzcv = [0] * 8, 0
    reg[:2] = vals
    for ins in prog:
        op, rd, rn, rm = ins[:4]
        cond = ins[5] if len(ins) > 5 else 0
        reg[rd], nzcv = NL.armv8_insn(op, reg[rd], reg[rn], reg[rm], 0, cond, nzcv)
    for r in range(2, 6):
        assert dec_word(ce, sk, ce.ce_reg_read(c, cid, r)) == reg[r], r


def test_serving_mix_levels_match_oracle(ce, ctx, keys, O, full_keys):
    """Four clients with their own keys; requests overlap on the GPU through
    the serving loop.  Sampled gates of every tick, each checked with its
    own client's oracle keys."""
    c, cid0 = ctx
    sk0, _ = keys
    clients = [(sk0, cid0, full_keys)]
    extra = []
    try:
        for k in range(3):
            seed = MASTER_SEED + 200 + k
            sk = ce.ce_secret_keygen(seed)
            cid = ce.ce_client_admit(c, ce.ce_cloud_keygen(sk, seed))
            extra.append(cid)
            clients.append((sk, cid, O.keygen(O.GATE_PARAMS, seed)))
        rng = np.random.default_rng(8)
        vals = {}
        for i, (sk, cid, _) in enumerate(clients):
            vals[cid] = [int(x) for x in rng.integers(0, 1 << W, 2)]
            for r, v in enumerate(vals[cid]):
                ce.ce_reg_write(c, cid, r, enc_word(ce, sk, v, 80 + i, 16 * r))
        ops = [("ADD", 2, 0, 1), ("SUB", 2, 0, 1), ("LSL", 2, 0, 1), ("CMP", 0, 0, 1)]
        ce.ce_trace_enable(c, 4, 4096)
        srv = ce.ce_server_create(c)
        try:
            tickets = [ce.ce_server_submit(srv, cid, ce.insn(*ops[i]))
                       for i, (_, cid, _) in enumerate(clients)]
            for t in tickets:
                ce.ce_server_wait(srv, t, 600 * 10**9)
        finally:
            ce.ce_server_destroy(srv)
        recs, seen = ce.ce_trace_read(c)
        ce.ce_trace_enable(c, 0)
        assert seen == len(recs) > 0
        assert len(set(recs["client"].tolist())) == 4, "not every client was sampled"
        assert oracle_check(O, {cid: ok for _, cid, ok in clients}, recs) == []
        for i, (sk, cid, _) in enumerate(clients[:3]):
            a, b = vals[cid]
            exp = NL.armv8(ops[i][0], a, b, W)
            assert dec_word(ce, sk, ce.ce_reg_read(c, cid, 2)) == exp
    finally:
        ce.ce_trace_enable(c, 0)
        for e in extra:
            ce.ce_client_evict(c, e)


def test_signed_multiplier_levels_match_oracle(ce, ctx, keys, O, full_keys):
    """16-bit SMULL (the full 32-bit signed product, §5 "Signed
    multiplication"): two sampled gates of every level against the oracle,
    and the decrypted product against signed semantics."""
    import torch
    c, cid = ctx
    sk, _ = keys
    a, b = 0x8003, 0x7FF1                      # negative times positive
    bits = [(a >> j) & 1 for j in range(W)] + [(b >> j) & 1 for j in range(W)]
    inp = np.stack([ce.ce_encrypt_bit(sk, x, 47, j) for j, x in enumerate(bits)])[None]
    d_out = torch.empty((1, 2 * W, 501), dtype=torch.int32, device="cuda")
    ce.ce_trace_enable(c, 2, 4096)
    try:
        ce.ce_unit_eval_device(c, cid, "SMULL", to_dev(inp.view(np.int32)), d_out, 1, 0)
        ce.ce_synchronize(c)
        recs, _ = ce.ce_trace_read(c)
    finally:
        ce.ce_trace_enable(c, 0)
    depth = ce.ce_unit_info("SMULL")["depth"]
    assert sorted(set(recs["tick"].tolist())) == list(range(depth))
    assert oracle_check(O, {cid: full_keys}, recs) == []
    out = d_out.cpu().numpy().view(np.uint32)[0]
    assert NL.from_bits([ce.ce_decrypt_bit(sk, x) for x in out]) == NL.armv8("SMULL", a, b, W)


@pytest.mark.parametrize("unit,pairs,per_level", [("ADD", 256, 6), ("MUL", 64, 4)])
def test_bench_configurations_match_oracle(ce, ctx, keys, O, full_keys, unit, pairs, per_level):
    """The bench's own workloads at full size — the 16-bit ADD on 256 operand
    pairs (49,664 bootstraps in 9 levels, the timed step) and the 16-bit MUL
    on 64 pairs — in the launch shapes the bench uses: sampled gates of every
    level against the oracle on the GPU's level inputs, and sampled sums and
    products against integer arithmetic."""
    import torch
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(1000 + pairs)
    a = rng.integers(0, 1 << W, pairs)
    b = rng.integers(0, 1 << W, pairs)
    inp = np.zeros((pairs, 2 * W, 501), np.uint32)
    for i in range(pairs):
        for j in range(W):
            inp[i, j] = ce.ce_encrypt_bit(sk, int(a[i] >> j) & 1, 60, 2 * W * i + j)
            inp[i, W + j] = ce.ce_encrypt_bit(sk, int(b[i] >> j) & 1, 60, 2 * W * i + W + j)
    d_out = torch.empty((pairs, W, 501), dtype=torch.int32, device="cuda")
    ce.ce_trace_enable(c, per_level, 4096)
    try:
        ce.ce_unit_eval_device(c, cid, unit, to_dev(inp.view(np.int32)), d_out, pairs, 0)
        ce.ce_synchronize(c)
        recs, seen = ce.ce_trace_read(c)
    finally:
        ce.ce_trace_enable(c, 0)
    depth = ce.ce_unit_info(unit)["depth"]
    assert seen == len(recs) == depth * per_level
    assert sorted(set(recs["tick"].tolist())) == list(range(depth))
    assert oracle_check(O, {cid: full_keys}, recs) == []
    out = d_out.cpu().numpy().view(np.uint32)
    for i in rng.choice(pairs, 8, replace=False):
        exp = NL.armv8(unit, int(a[i]), int(b[i]), W)
        assert dec_word(ce, sk, out[i]) == exp, (unit, i)


def test_tree_multiplier_levels_match_oracle(ce, ctx, keys, O, full_keys):
    """MUL_TREE (column compression, 697 bootstraps in 18 levels) on two
    operand pairs: three sampled gates of every level, full-adder MUX
    carries included, against the oracle on the GPU's level inputs; the
    products against integer arithmetic."""
    import torch
    c, cid = ctx
    sk, _ = keys
    a, b = np.array([0xBEEF, 0xFFFF]), np.array([0x7A31, 0xFFFF])
    inp = np.stack([np.concatenate([enc_word(ce, sk, int(a[i]), 70 + i, 0),
                                    enc_word(ce, sk, int(b[i]), 72 + i, 16)]) for i in range(2)])
    d_out = torch.empty((2, W, 501), dtype=torch.int32, device="cuda")
    ce.ce_trace_enable(c, 3, 4096)
    try:
        ce.ce_unit_eval_device(c, cid, "MUL_TREE", to_dev(inp.view(np.int32)), d_out, 2, 0)
        ce.ce_synchronize(c)
        recs, seen = ce.ce_trace_read(c)
    finally:
        ce.ce_trace_enable(c, 0)
    depth = ce.ce_unit_info("MUL_TREE")["depth"]
    assert seen == len(recs) > 0
    assert sorted(set(recs["tick"].tolist())) == list(range(depth))
    assert (recs["op"] == 10).any(), "no MUX (full-adder carry) was sampled"
    assert oracle_check(O, {cid: full_keys}, recs) == []
    out = d_out.cpu().numpy().view(np.uint32)
    for i in range(2):
        assert dec_word(ce, sk, out[i]) == (int(a[i]) * int(b[i])) & 0xFFFF
