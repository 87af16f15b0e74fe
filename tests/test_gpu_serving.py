"""Serving loop: requests from several clients (each with its own keys) are
batched continuously; a request's result is bit-identical alone and in the
mix; each client's requests run in order; admission respects the HBM budget;
bad requests are errors."""
import numpy as np
import pytest

from gpu_common import MASTER_SEED, ce, ctx, keys  # noqa: F401

pytestmark = pytest.mark.gpu
W = 16


def enc_word(ce, sk, v, seed, base):
    return np.stack([ce.ce_encrypt_bit(sk, (v >> j) & 1, seed, base + j) for j in range(W)])


def dec_word(ce, sk, bits):
    return sum(ce.ce_decrypt_bit(sk, bits[j]) << j for j in range(W))


@pytest.fixture(scope="module")
def clients(ce, ctx, keys):
    """The shared client plus three more with their own key sets."""
    c, cid = ctx
    out = [(keys[0], cid)]
    extra = []
    for k in range(3):
        sk = ce.ce_secret_keygen(MASTER_SEED + 100 + k)
        ck = ce.ce_cloud_keygen(sk, MASTER_SEED + 100 + k)
        extra.append(ce.ce_client_admit(c, ck))
        out.append((sk, extra[-1]))
    yield out
    for e in extra:
        ce.ce_client_evict(c, e)


def test_alone_equals_in_mix(ce, ctx, clients):
    c, _ = ctx
    rng = np.random.default_rng(5)
    vals = {i: [int(x) for x in rng.integers(0, 1 << W, 4)] for i in range(len(clients))}
    regs = {i: [enc_word(ce, sk, v, 60 + i, 16 * r) for r, v in enumerate(vals[i])]
            for i, (sk, _) in enumerate(clients)}

    def load(i):
        for r, bits in enumerate(regs[i]):
            ce.ce_reg_write(c, clients[i][1], r, bits)

    sk0, cid0 = clients[0]
    add = ce.insn("ADD", 2, 0, 1)
    # alone
    load(0)
    srv = ce.ce_server_create(c)
    t = ce.ce_server_submit(srv, cid0, add)
    ce.ce_server_wait(srv, t, 600 * 10**9)
    alone = ce.ce_reg_read(c, cid0, 2)
    # in a mix: other clients' MUL/SUB/ADD requests, the same ADD submitted mid-stream
    for i in range(4):
        load(i)
    ops = [("MUL", 3, 0, 1), ("SUB", 3, 1, 0), ("ADD", 3, 2, 1), ("LSL", 3, 0, 1)]
    tickets = []
    for k in range(6):
        i = 1 + k % 3
        tickets.append(ce.ce_server_submit(srv, clients[i][1], ce.insn(*ops[k % 4])))
        if k == 2:
            t0 = ce.ce_server_submit(srv, cid0, add)
    for t in tickets + [t0]:
        ce.ce_server_wait(srv, t, 600 * 10**9)
    stats = ce.ce_server_stats(srv)
    ce.ce_server_destroy(srv)
    mixed = ce.ce_reg_read(c, cid0, 2)
    assert (alone == mixed).all(), "result differs alone vs in the mix"
    assert dec_word(ce, sk0, mixed) == (vals[0][0] + vals[0][1]) & 0xFFFF
    assert stats["ticks"] > 0 and stats["bootstraps"] > 0


def test_client_requests_run_in_order(ce, ctx, clients):
    c, _ = ctx
    sk, cid = clients[1]
    a, b = 40000, 30000
    ce.ce_reg_write(c, cid, 0, enc_word(ce, sk, a, 70, 0))
    ce.ce_reg_write(c, cid, 1, enc_word(ce, sk, b, 70, 16))
    srv = ce.ce_server_create(c, 2)
    t1 = ce.ce_server_submit(srv, cid, ce.insn("ADD", 2, 0, 1))      # r2 = a + b
    t2 = ce.ce_server_submit(srv, cid, ce.insn("SUB", 3, 2, 0))      # r3 = r2 - a = b
    t3 = ce.ce_server_submit(srv, cid, ce.insn("MOV", 4, 3))
    for t in (t1, t2, t3):
        ce.ce_server_wait(srv, t, 600 * 10**9)
    info = [ce.ce_server_poll(srv, t) for t in (t1, t2, t3)]
    ce.ce_server_destroy(srv)
    # start_ns is when the host enqueues a request's first level: it may
    # precede the previous request's GPU completion (stream order still runs
    # it after).  Completions are in submission order, and the dependent SUB
    # below reads the ADD's result.
    assert info[0]["done_ns"] <= info[1]["done_ns"] <= info[2]["done_ns"]
    assert info[0]["start_ns"] <= info[1]["start_ns"] <= info[2]["start_ns"]
    assert dec_word(ce, sk, ce.ce_reg_read(c, cid, 2)) == (a + b) & 0xFFFF
    assert dec_word(ce, sk, ce.ce_reg_read(c, cid, 4)) == b


def test_server_errors(ce, ctx, clients):
    c, _ = ctx
    srv = ce.ce_server_create(c)
    with pytest.raises(ce.CeError) as ei:
        ce.ce_server_submit(srv, 12345, ce.insn("ADD", 0, 1, 2))
    assert ei.value.code == -6
    with pytest.raises(ce.CeError) as ei:
        ce.ce_server_submit(srv, clients[0][1], ce.insn("ADD", 8, 1, 2))
    assert ei.value.code == -1
    with pytest.raises(ce.CeError) as ei:
        ce.ce_server_wait(srv, 999999)
    assert ei.value.code == -6
    ce.ce_server_destroy(srv)


def test_admission_by_hbm_budget(ce, keys):
    fp = ce.ce_client_footprint_bytes()
    small = ce.ce_create(0, int(fp * 1.5))
    try:
        ce.ce_client_admit(small, keys[1])
        with pytest.raises(ce.CeError) as ei:
            ce.ce_client_admit(small, keys[1])
        assert ei.value.code == -3
    finally:
        small.close()


def test_evict_refused_while_requests_pending(ce, ctx):
    """Evicting a client whose request a serving loop still holds is refused
    on the host (CE_EINVAL) before anything is freed; once the request is
    done the eviction goes through."""
    c, _ = ctx
    seed = MASTER_SEED + 300
    sk = ce.ce_secret_keygen(seed)
    cid = ce.ce_client_admit(c, ce.ce_cloud_keygen(sk, seed))
    ce.ce_reg_write(c, cid, 0, enc_word(ce, sk, 50000, 90, 0))
    ce.ce_reg_write(c, cid, 1, enc_word(ce, sk, 7, 90, 16))
    srv = ce.ce_server_create(c)
    try:
        t = ce.ce_server_submit(srv, cid, ce.insn("UDIV", 2, 0, 1))   # ~0.7 s on the GPU
        with pytest.raises(ce.CeError) as ei:
            ce.ce_client_evict(c, cid)
        assert ei.value.code == -1
        ce.ce_server_wait(srv, t, 600 * 10**9)
    finally:
        ce.ce_server_destroy(srv)
    assert dec_word(ce, sk, ce.ce_reg_read(c, cid, 2)) == 50000 // 7
    ce.ce_client_evict(c, cid)
    with pytest.raises(ce.CeError) as ei:
        ce.ce_reg_read(c, cid, 2)
    assert ei.value.code == -6
