"""Encrypted register programs (ce_exec / ce_exec_multi) against a plaintext
model of the same 16-bit ARM-subset machine; several programs and two
clients advance together; malformed programs, unknown clients and the host
timeout are errors, not crashes."""
import numpy as np
import pytest

from gpu_common import MASTER_SEED, ce, ctx, keys  # noqa: F401
from oracle import netlists as NL

pytestmark = pytest.mark.gpu
W, M = 16, 0xFFFF


def run_plain(prog, regs, nzcv=0):
    regs = list(regs)
    for op, rd, rn, rm, imm, cond in prog:
        regs[rd], nzcv = NL.armv8_insn(op, regs[rd], regs[rn], regs[rm], imm, cond, nzcv, W)
    return regs, nzcv


def random_program(rng, length):
    ops = ["ADD", "SUB", "AND", "ORR", "LSL", "LSL_IMM", "CMP", "CSEL", "MOV", "MOV_IMM", "LSR",
           "ASR", "LSR_IMM", "ASR_IMM", "EOR", "ORN", "MVN", "AND_IMM", "ORR_IMM", "EOR_IMM",
           "BFC", "BFI", "RBIT", "REV"]
    prog = [("CMP", 0, 1, 2, 0, 0)]           # flags defined before any CSEL
    while len(prog) < length:
        op = ops[rng.integers(len(ops))]
        prog.append((op, int(rng.integers(8)), int(rng.integers(8)), int(rng.integers(8)),
                     int(rng.integers(256)), int(rng.integers(14))))
    return prog


def load_regs(ce, c, cid, sk, vals, seed):
    for r, v in enumerate(vals):
        bits = np.stack([ce.ce_encrypt_bit(sk, (v >> j) & 1, seed, 16 * r + j) for j in range(W)])
        ce.ce_reg_write(c, cid, r, bits)


def read_regs(ce, c, cid, sk):
    return [NL.from_bits([ce.ce_decrypt_bit(sk, x) for x in ce.ce_reg_read(c, cid, r)])
            for r in range(8)]


@pytest.fixture(scope="module")
def second_client(ce, ctx):
    c, _ = ctx
    sk2 = ce.ce_secret_keygen(MASTER_SEED + 1)
    ck2 = ce.ce_cloud_keygen(sk2, MASTER_SEED + 1)
    cid2 = ce.ce_client_admit(c, ck2)
    yield sk2, cid2
    ce.ce_client_evict(c, cid2)


def test_programs_two_clients(ce, ctx, keys, second_client):
    c, cid = ctx
    sk, _ = keys
    sk2, cid2 = second_client
    rng = np.random.default_rng(2021)
    # one program per client (each client has one register file)
    progs = [random_program(rng, int(rng.integers(8, 17))) for _ in range(2)]
    init = [[int(x) for x in rng.integers(0, 1 << W, 8)] for _ in range(2)]
    load_regs(ce, c, cid, sk, init[0], 40)
    load_regs(ce, c, cid2, sk2, init[1], 41)
    ce.ce_exec_multi(c, [cid, cid2], [[ce.insn(*i) for i in p] for p in progs])
    for (sk_, cid_), p, r0 in zip(((sk, cid), (sk2, cid2)), progs, init):
        exp_regs, exp_nzcv = run_plain(p, r0)
        assert read_regs(ce, c, cid_, sk_) == exp_regs
        flags = [ce.ce_decrypt_bit(sk_, x) for x in ce.ce_flags_read(c, cid_)]
        assert flags == [(exp_nzcv >> k) & 1 for k in range(4)]


def test_many_clients_in_one_level_equal_each_alone(ce, ctx, keys):
    """Twenty clients run one ADD at once: the engine's first level holds
    640 gates (more than one round of four-gate groups over the SMs), so the
    blind rotation runs as whole rounds plus a tail launch that looks each
    group's key up by its position in the batch.  Every client's result
    register must equal, word for word, the same instruction run for that
    client alone, and decrypt to the plaintext sum."""
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(77)
    clients = [(sk, cid)]
    extra = []
    try:
        for i in range(19):
            ski = ce.ce_secret_keygen(MASTER_SEED + 200 + i)
            cidi = ce.ce_client_admit(c, ce.ce_cloud_keygen(ski, MASTER_SEED + 200 + i))
            extra.append(cidi)
            clients.append((ski, cidi))
        vals = [[int(x) for x in rng.integers(0, 1 << W, 2)] for _ in clients]
        prog = [ce.insn("ADD", 2, 0, 1)]

        def load(k):
            ski, cidi = clients[k]
            for r in range(2):
                ce.ce_reg_write(c, cidi, r, np.stack(
                    [ce.ce_encrypt_bit(ski, (vals[k][r] >> j) & 1, 90 + k, 16 * r + j)
                     for j in range(W)]))

        for k in range(len(clients)):
            load(k)
        ce.ce_exec_multi(c, [x[1] for x in clients], [prog] * len(clients))
        together = [ce.ce_reg_read(c, x[1], 2).copy() for x in clients]
        for k, (ski, cidi) in enumerate(clients):
            load(k)
            ce.ce_exec(c, cidi, prog)
            alone = ce.ce_reg_read(c, cidi, 2)
            assert (alone == together[k]).all(), k
            got = NL.from_bits([ce.ce_decrypt_bit(ski, x) for x in alone])
            assert got == (vals[k][0] + vals[k][1]) & 0xFFFF
    finally:
        for cidi in extra:
            ce.ce_client_evict(c, cidi)


def test_every_instruction(ce, ctx, keys):
    """Each of the machine's register instructions at least once, in a random
    order with random operands, against the plaintext model."""
    c, cid = ctx
    sk, _ = keys
    rng = np.random.default_rng(2022)
    # MUL, UDIV: test below; branches: ce_exec_branching (test below)
    ops = [o for o in ce.OPCODES if o not in ("MUL", "UDIV", "BCOND", "B")]
    prog = [("CMP", 0, 1, 2, 0, 0)]
    for op in rng.permutation(ops + ops):
        prog.append((str(op), int(rng.integers(8)), int(rng.integers(8)), int(rng.integers(8)),
                     int(rng.integers(256)), int(rng.integers(14))))
    init = [int(x) for x in rng.integers(0, 1 << W, 8)]
    load_regs(ce, c, cid, sk, init, 43)
    ce.ce_exec(c, cid, [ce.insn(*i) for i in prog])
    exp_regs, exp_nzcv = run_plain(prog, init)
    assert read_regs(ce, c, cid, sk) == exp_regs
    flags = [ce.ce_decrypt_bit(sk, x) for x in ce.ce_flags_read(c, cid)]
    assert flags == [(exp_nzcv >> k) & 1 for k in range(4)]


def test_low_latency_instruction_circuits(ce, ctx, keys):
    """ADD, SUB, MUL and UDIV on the MUX-carry adders and the tree
    multiplier (ce_set_instruction_circuits): the plaintext machine's
    registers, with the program set planned and replayed as a graph and run
    eagerly."""
    c, cid = ctx
    sk, _ = keys
    init = [1234, 56, 0xFFFF, 7, 65535, 3, 0x8000, 9]
    prog = [("ADD", 2, 0, 1, 0, 0), ("SUB", 3, 1, 0, 0, 0), ("MUL", 5, 0, 1, 0, 0),
            ("ADD", 6, 4, 6, 0, 0), ("MUL", 7, 2, 3, 0, 0), ("SUB", 1, 7, 2, 0, 0),
            ("UDIV", 4, 4, 1, 0, 0)]
    exp = run_plain(prog, init)[0]
    ce.ce_set_instruction_circuits(c, True)
    try:
        for graphs in (True, False):
            ce.ce_set_unit_graphs(c, graphs)
            load_regs(ce, c, cid, sk, init, 44)
            ce.ce_exec(c, cid, [ce.insn(*i) for i in prog])
            assert read_regs(ce, c, cid, sk) == exp
    finally:
        ce.ce_set_unit_graphs(c, True)
        ce.ce_set_instruction_circuits(c, False)


def test_mul_udiv_program(ce, ctx, keys):
    c, cid = ctx
    sk, _ = keys
    init = [1234, 56, 0, 7, 65535, 3, 0, 9]
    prog = [("MUL", 2, 0, 1, 0, 0), ("UDIV", 6, 4, 3, 0, 0), ("UDIV", 7, 0, 6, 0, 0)]
    load_regs(ce, c, cid, sk, init, 42)
    ce.ce_exec(c, cid, [ce.insn(*i) for i in prog])
    assert read_regs(ce, c, cid, sk) == run_plain(prog, init)[0]


def test_program_errors(ce, ctx):
    c, cid = ctx
    with pytest.raises(ce.CeError) as ei:
        ce.ce_exec(c, cid, [ce.insn("ADD", 9, 0, 0)])          # register out of range
    assert ei.value.code == -1
    with pytest.raises(ce.CeError) as ei:
        ce.ce_exec(c, 999, [ce.insn("ADD", 0, 0, 0)])
    assert ei.value.code == -6
    with pytest.raises(ce.CeError) as ei:                       # host-side timeout
        ce.ce_exec(c, cid, [ce.insn("ADD", 0, 1, 2)] * 4, timeout_ns=1)
    assert ei.value.code == -4
    ce.ce_synchronize(c)


def run_plain_branching(prog, regs, max_steps=10000):
    """The plaintext machine with a cleartext program counter (§6 "Branch")."""
    regs, nzcv, pc, steps = list(regs), 0, 0, 0
    while pc < len(prog):
        op, rd, rn, rm, imm, cond = prog[pc]
        steps += 1
        assert steps <= max_steps
        if op == "B":
            pc = imm
        elif op == "BCOND":
            pc = imm if NL.armv8("CSEL", 1, 0, W, cond, nzcv) else pc + 1
        else:
            regs[rd], nzcv = NL.armv8_insn(op, regs[rd], regs[rn], regs[rm], imm, cond, nzcv, W)
            pc += 1
    return regs, nzcv, steps


def test_branching_loop_resolved_by_the_key_owner(ce, ctx, keys):
    """A counted loop closed by B.NE, an unconditional branch over dead code,
    and the signed/unsigned high-half multiplies; the branch decisions are
    made by a callback that decrypts the encrypted NZCV with the secret key
    (the client side of §6's branch resolution)."""
    c, cid = ctx
    sk, _ = keys
    prog = [("MOV_IMM", 3, 0, 0, 1, 0), ("MOV_IMM", 4, 0, 0, 0, 0), ("MOV_IMM", 2, 0, 0, 0, 0),
            ("ADD", 2, 2, 0, 0, 0),            # 3: loop body
            ("SUB", 1, 1, 3, 0, 0),
            ("CMP", 0, 1, 4, 0, 0),
            ("BCOND", 0, 0, 0, 3, 1),          # B.NE 3
            ("SMULH", 5, 2, 0, 0, 0),
            ("B", 0, 0, 0, 10, 0),
            ("MOV_IMM", 6, 0, 0, 77, 0),       # skipped
            ("UMULH", 7, 0, 2, 0, 0)]
    init = [0xC123, 3, 0, 0, 0, 0, 0x5555, 0]
    load_regs(ce, c, cid, sk, init, 44)
    asked = []

    def decide(client, cond, nzcv):
        f = [ce.ce_decrypt_bit(sk, x) for x in nzcv]
        asked.append((client, cond))
        return NL.armv8("CSEL", 1, 0, W, cond, f[0] | f[1] << 1 | f[2] << 2 | f[3] << 3) == 1

    steps = ce.ce_exec_branching(c, cid, [ce.insn(*i) for i in prog], decide, max_steps=100)
    exp_regs, exp_nzcv, exp_steps = run_plain_branching(prog, init)
    assert steps == exp_steps
    assert asked == [(cid, 1)] * 3                      # three B.NE decisions
    assert read_regs(ce, c, cid, sk) == exp_regs
    assert exp_regs[6] == 0x5555                          # the dead code stayed dead


def test_branching_errors(ce, ctx):
    c, cid = ctx
    with pytest.raises(ce.CeError) as ei:                   # ce_exec runs no branches
        ce.ce_exec(c, cid, [ce.insn("B", imm=1)])
    assert ei.value.code == -1
    with pytest.raises(ce.CeError) as ei:                   # an endless loop hits the step limit
        ce.ce_exec_branching(c, cid, [ce.insn("B", imm=0)], lambda *a: True, max_steps=50)
    assert ei.value.code == -4
    with pytest.raises(ce.CeError) as ei:                   # target beyond the end
        ce.ce_exec_branching(c, cid, [ce.insn("B", imm=5)], lambda *a: True)
    assert ei.value.code == -1


def test_program_graph_replay_equals_eager(ce, ctx, keys, second_client):
    """Two programs on two clients (§4 "Data Processing" register machines)
    run three times from the same encrypted registers: eager ticks, then
    planned and captured as a CUDA graph, then replayed; every register and
    flag ciphertext is identical across the three, and decrypts to the
    plaintext machine's result."""
    c, cid = ctx
    sk, _ = keys
    sk2, cid2 = second_client
    rng = np.random.default_rng(2023)
    progs = [random_program(rng, 14), random_program(rng, 10)]
    init = [[int(x) for x in rng.integers(0, 1 << W, 8)] for _ in range(2)]

    def run(graphs):
        load_regs(ce, c, cid, sk, init[0], 45)
        load_regs(ce, c, cid2, sk2, init[1], 46)
        ce.ce_set_unit_graphs(c, graphs)
        try:
            ce.ce_exec_multi(c, [cid, cid2], [[ce.insn(*i) for i in p] for p in progs])
        finally:
            ce.ce_set_unit_graphs(c, True)
        return [np.concatenate([ce.ce_reg_read(c, x, r) for r in range(8)] +
                               [ce.ce_flags_read(c, x)]) for x in (cid, cid2)]

    eager = run(False)
    first = run(True)
    replay = run(True)
    for a, b, d in zip(eager, first, replay):
        assert (a == b).all() and (a == d).all()
    for (s, x), p, v in zip(((sk, cid), (sk2, cid2)), progs, init):
        exp_regs, exp_nzcv = run_plain(p, v)
        assert read_regs(ce, c, x, s) == exp_regs
        assert [ce.ce_decrypt_bit(s, f) for f in ce.ce_flags_read(c, x)] == \
            [(exp_nzcv >> k) & 1 for k in range(4)]
