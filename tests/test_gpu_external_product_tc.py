"""Blind rotation with the Toeplitz external product on the tensor cores,
against the plain CPU oracle and against the transform form.

Every CMux step of a bootstrap (§3 "TFHE Library": n = 500 external
products) runs as one [gates x 6144 digits] x [6144 x 2048] product with the
key's negacyclic Toeplitz blocks, key words in four balanced byte limbs and
digits in two balanced 5-bit limbs (fp16 operands, exact fp32 sums).
Ciphertexts must equal the oracle word for word (all of them for small
batches, sampled ones for large), and the transform form on every output:
across gate tiles of 128 with ragged tails, stream-K ranges that split
tiles between CTAs (partial sums added atomically: 1, 2, 3 and 10 tiles)
and ranges of whole tiles (19 tiles, two per CTA), zero rotations, MUX
pairs, and the levels of a 16-bit unit run by the netlist engine.
"""
import numpy as np
import pytest

from gpu_common import (ce, ctx, keys, encrypt_bits, random_ciphertexts,  # noqa: F401
                        run_gates_device, to_dev)

pytestmark = pytest.mark.gpu


def with_form(ce, c, form, fn):
    ce.ce_set_external_product_form(c, form)
    try:
        return fn()
    finally:
        ce.ce_set_external_product_form(c, 0)


def test_truth_tables_tensor_form(ce, ctx, keys, O, full_keys):
    c, _ = ctx
    sk, _ = keys
    ops, bits = [], []
    for op in ("NAND", "AND", "OR", "XOR", "XNOR", "NOR", "ANDNY", "ORYN"):
        for a in (0, 1):
            for b in (0, 1):
                ops.append(O.GATE_ID[op])
                bits.append((a, b))
    bits = np.array(bits)
    ca = encrypt_bits(ce, sk, bits[:, 0], 31)
    cb = encrypt_bits(ce, sk, bits[:, 1], 32)
    got = with_form(ce, c, 1, lambda: run_gates_device(ce, ctx, ops, ca, cb))
    exp = O.gates(full_keys, ops, ca, cb)
    assert (got == exp).all()
    for i, op in enumerate(ops):
        assert ce.ce_decrypt_bit(sk, got[i]) == O.TRUTH[O.GATES[op]](*bits[i])


def test_zero_rotations_and_trivial_inputs_tensor_form(ce, ctx, O, full_keys):
    """abar_i = 0 for many i (the CMux step adds zero digits) and trivial
    ciphertexts."""
    c, _ = ctx
    rng = np.random.default_rng(41)
    a, b = random_ciphertexts(rng, 5), random_ciphertexts(rng, 5)
    a[0, :500] = 0
    b[0, :500] = 0
    a[1, ::2] = 0x000FFFFF
    b[1, ::3] = 0xFFF00000
    a[2, :500] = 0
    b[2, :500] = 0
    a[2, 500], b[2, 500] = 0x20000000, 0xE0000000
    a[3, :500] = 0x40000000         # rotations by exactly N (X^N = -1)
    b[3, :500] = 0
    ops = [0, 1, 2, 3, 4]
    got = with_form(ce, c, 1, lambda: run_gates_device(ce, ctx, ops, a, b))
    assert (got == O.gates(full_keys, ops, a, b)).all()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 300, 1201, 2432])
def test_tensor_form_equals_transform_form_and_oracle(ce, ctx, O, full_keys, n):
    c, _ = ctx
    rng = np.random.default_rng(4000 + n)
    ops = rng.integers(0, 10, n)
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    got = with_form(ce, c, 1, lambda: run_gates_device(ce, ctx, ops, a, b))
    ref = run_gates_device(ce, ctx, ops, a, b)
    assert (got == ref).all()
    idx = np.unique(np.concatenate([rng.choice(n, min(n, 2), replace=False), [0, n - 1]]))
    assert (got[idx] == O.gates(full_keys, ops[idx], a[idx], b[idx])).all()


def test_mux_tensor_form(ce, ctx, keys, O, full_keys):
    import torch
    c, cid = ctx
    sk, _ = keys
    sel = np.array([(i >> 2) & 1 for i in range(8)])
    x = np.array([(i >> 1) & 1 for i in range(8)])
    y = np.array([i & 1 for i in range(8)])
    ca, cb, cc = (encrypt_bits(ce, sk, v, s) for v, s in ((sel, 51), (x, 52), (y, 53)))
    n = len(sel)

    def run():
        out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
        ce.ce_mux_batch_device(c, cid, to_dev(ca.view(np.int32)), to_dev(cb.view(np.int32)),
                               to_dev(cc.view(np.int32)), out, n)
        ce.ce_synchronize(c)
        return out.cpu().numpy().view(np.uint32)

    got = with_form(ce, c, 1, run)
    assert (got == run()).all()
    for i in range(n):
        assert ce.ce_decrypt_bit(sk, got[i]) == (x[i] if sel[i] else y[i])
        if i < 2:
            assert (got[i] == O.mux(full_keys, ca[i], cb[i], cc[i])).all()


@pytest.mark.parametrize("pairs", [3, 64])
def test_unit_add_tensor_form(ce, ctx, keys, pairs):
    import torch
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(60 + pairs)
    bits = rng.integers(0, 2, (pairs, 32))
    ct = encrypt_bits(ce, sk, bits.reshape(-1), 960 + pairs).reshape(pairs, 32, 501)
    d_in = to_dev(ct.view(np.int32))

    def run():
        out = torch.empty((pairs, 16, 501), dtype=torch.int32, device="cuda")
        ce.ce_unit_eval_device(c, cid, "ADD", d_in, out, pairs, 0, torch.cuda.current_stream())
        ce.ce_synchronize(c)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    got = with_form(ce, c, 1, run)
    assert (got == run()).all()
    for i in range(pairs):
        av = sum(int(bits[i, j]) << j for j in range(16))
        bv = sum(int(bits[i, 16 + j]) << j for j in range(16))
        res = sum(ce.ce_decrypt_bit(sk, got[i, j].view(np.uint32)) << j for j in range(16))
        assert res == (av + bv) & 0xFFFF


def test_launch_count_of_tensor_form(ce, ctx):
    """Linear combination, 1 + 2 x 500 blind-rotation launches, rounding and
    key switch (tensor key switch from 32 outputs)."""
    c, _ = ctx
    rng = np.random.default_rng(70)
    n = 40
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    with_form(ce, c, 1, lambda: run_gates_device(ce, ctx, np.zeros(n, np.int64), a, b))
    ce.ce_set_external_product_form(c, 1)
    try:
        run_gates_device(ce, ctx, np.zeros(n, np.int64), a, b)
        assert ce.ce_last_launch_count(c) == 1 + 1001 + 2
    finally:
        ce.ce_set_external_product_form(c, 0)


def test_form_rejects_bad_values(ce, ctx):
    c, _ = ctx
    for bad in (-1, 2):
        with pytest.raises(Exception):
            ce.ce_set_external_product_form(c, bad)


def test_profile_times_the_mma_launches(ce, ctx):
    """Profiling kind 3: one event pair per CMux step's MMA launch."""
    c, _ = ctx
    rng = np.random.default_rng(71)
    n = 40
    a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
    ce.ce_set_external_product_form(c, 1)
    try:
        ce.ce_profile_enable(c, True)
        run_gates_device(ce, ctx, np.zeros(n, np.int64), a, b)
        prof = ce.ce_profile_read(c)
    finally:
        ce.ce_profile_enable(c, False)
        ce.ce_set_external_product_form(c, 0)
    ms, cnt = prof["external_product_mma"]
    assert cnt == 500
    assert 0 < ms <= prof["blind_rotate"][0]


def test_tensor_key_over_budget_is_refused(ce, keys):
    """The tensor form's key (783,360,000 B) is built on first use and counted
    against the HBM budget: a context with room for the client but not for
    that key refuses with CE_EADMIT and keeps working in the transform form."""
    import torch
    from paper_2101_03403_gb300 import CeError
    sk, ck = keys
    c = ce.ce_create(0, ce.ce_client_footprint_bytes() + (100 << 20))
    try:
        cid = ce.ce_client_admit(c, ck)
        rng = np.random.default_rng(80)
        n = 3
        a, b = random_ciphertexts(rng, n), random_ciphertexts(rng, n)
        ops = np.array([0, 1, 2], np.uint8)
        ce.ce_set_external_product_form(c, 1)
        out = torch.empty((n, 501), dtype=torch.int32, device="cuda")
        with pytest.raises(CeError) as ex:
            ce.ce_gates_batch_device(c, cid, to_dev(ops), to_dev(a.view(np.int32)),
                                     to_dev(b.view(np.int32)), out, n)
        assert ex.value.code == -3                      # CE_EADMIT
        ce.ce_set_external_product_form(c, 0)
        ce.ce_gates_batch_device(c, cid, to_dev(ops), to_dev(a.view(np.int32)),
                                 to_dev(b.view(np.int32)), out, n)
        ce.ce_synchronize(c)
        assert out.cpu().numpy().view(np.uint32).shape == (n, 501)
    finally:
        c.close()


def test_programs_of_two_clients_in_tensor_form(ce, ctx, keys):
    """Engine ticks that mix clients run the transform form (each gate group
    with its own key); single-client ticks the tensor form: the registers
    after the programs are identical to a run entirely in the transform form."""
    c, cid = ctx
    sk, ck = keys
    sk2 = ce.ce_secret_keygen(777)
    cid2 = ce.ce_client_admit(c, ce.ce_cloud_keygen(sk2, 777))
    try:
        rng = np.random.default_rng(81)
        regs = {}
        for cl, key in ((cid, sk), (cid2, sk2)):
            for r in range(3):
                v = int(rng.integers(0, 1 << 16))
                bits = [ce.ce_encrypt_bit(key, (v >> j) & 1, 90 + r, cl * 16 + j)
                        for j in range(16)]
                regs[(cl, r)] = np.stack(bits)
        progs = [[ce.insn("ADD", 2, 0, 1), ce.insn("AND", 0, 2, 1)],
                 [ce.insn("SUB", 2, 1, 0)]]
        results = []
        for form in (1, 0):
            for (cl, r), v in regs.items():
                ce.ce_reg_write(c, cl, r, v)
            ce.ce_set_external_product_form(c, form)
            try:
                ce.ce_exec_multi(c, [cid, cid2], progs)
                ce.ce_synchronize(c)
            finally:
                ce.ce_set_external_product_form(c, 0)
            results.append([ce.ce_reg_read(c, cl, r) for cl in (cid, cid2) for r in range(3)])
        for x, y in zip(*results):
            assert (x == y).all()
    finally:
        ce.ce_client_evict(c, cid2)
