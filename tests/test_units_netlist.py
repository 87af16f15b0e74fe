"""Functional-unit netlists: the oracle's construction (oracle/netlists.py)
checked exhaustively against ARMv8 semantics at width 8 and on random
16-bit operands, gate counts against the paper's structure, and the
library's independently built netlists equal to the oracle's gate for gate."""
import numpy as np
import pytest

from oracle import netlists as NL

UNITS = ["ADD", "ADD_RIPPLE", "SUB", "AND", "ORR", "LSL", "MUL", "UDIV", "CMP", "LSR", "ASR",
         "EOR", "ORN", "ADDS", "SUBS", "SMULL", "UMULL", "ADD_MUX", "SUB_MUX", "MUL_TREE",
         "UDIV_MUX"]


def eval_vec(net, inputs):
    """Plaintext evaluation on arrays of input bits (one array per input)."""
    n = len(inputs[0])
    val = [np.asarray(x, np.uint8) for x in inputs] + [None] * (len(net.levels) - net.n_inputs)
    zero = np.zeros(n, np.uint8)

    def rd(r):
        v = zero if r[0] < 0 else val[r[0]]
        return 1 - v if r[1] else v

    for op, a, b, c, out, _ in net.by_level():
        if op == NL.MUX:
            val[out] = np.where(rd(a) == 1, rd(b), rd(c)).astype(np.uint8)
        else:
            val[out] = np.asarray(NL.GATE_FN[op](rd(a).astype(np.int64), rd(b).astype(np.int64)),
                                  np.uint8)
    return [rd(r) for r in net.outputs]


def check_unit(unit, w, a, b, cond=0, nzcv=None):
    net = NL.build(unit, w, cond)
    ins = [(a >> i) & 1 for i in range(w)] + [(b >> i) & 1 for i in range(w)]
    if unit == "CSEL":
        ins += [(nzcv >> i) & 1 for i in range(4)]
    outs = eval_vec(net, ins)
    if unit == "CMP":
        exp = np.array([NL.armv8(unit, int(x), int(y), w) for x, y in zip(a, b)])
        for k in range(4):
            assert (outs[k] == exp[:, k]).all(), (unit, k)
    elif unit in ("ADDS", "SUBS"):
        exp = np.array([NL.armv8(unit, int(x), int(y), w) for x, y in zip(a, b)])
        got = sum(outs[i].astype(np.int64) << i for i in range(w))
        assert (got == exp[:, 0]).all(), unit
        for k in range(4):
            assert (outs[w + k] == exp[:, 1 + k]).all(), (unit, k)
    elif unit in ("SMULL", "UMULL"):           # 2w-bit products (Python integers)
        got = [sum(int(outs[i][k]) << i for i in range(2 * w)) for k in range(len(a))]
        exp = [NL.armv8(unit, int(x), int(y), w) for x, y in zip(a, b)]
        bad = [k for k in range(len(a)) if got[k] != exp[k]]
        assert not bad, (unit, int(a[bad[0]]), int(b[bad[0]]), got[bad[0]], exp[bad[0]])
    else:
        got = sum(outs[i].astype(np.int64) << i for i in range(w))
        if unit == "CSEL":
            exp = np.array([NL.armv8(unit, int(x), int(y), w, cond, int(f))
                            for x, y, f in zip(a, b, nzcv)])
        else:
            exp = np.array([NL.armv8(unit, int(x), int(y), w) for x, y in zip(a, b)])
        bad = np.nonzero(got != exp)[0]
        assert len(bad) == 0, (unit, int(a[bad[0]]), int(b[bad[0]]), int(got[bad[0]]))


@pytest.mark.parametrize("unit", UNITS)
def test_exhaustive_width8(unit):
    a, b = np.meshgrid(np.arange(256), np.arange(256))
    check_unit(unit, 8, a.ravel(), b.ravel())


@pytest.mark.parametrize("unit", UNITS)
def test_random_width16(unit):
    rng = np.random.default_rng(16)
    a = rng.integers(0, 1 << 16, 4000)
    b = rng.integers(0, 1 << 16, 4000)
    b[:40] = 0
    b[40:80] = a[40:80]
    a[80:120] = 0xFFFF
    check_unit(unit, 16, a, b)


@pytest.mark.parametrize("unit", UNITS)
def test_random_width32(unit):
    rng = np.random.default_rng(32)
    n = 600 if unit.startswith("UDIV") else 2000
    a = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.int64)
    b = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.int64)
    b[:20] = 0
    b[20:40] = a[20:40]
    a[40:60] = 0xFFFFFFFF
    b[60:120] = rng.integers(0, 64, 60)           # every shift amount mod 32
    if unit.startswith("UDIV"):
        b[120:200] = rng.integers(1, 1 << 16, 80)  # quotients of every size
    check_unit(unit, 32, a, b)


def test_right_shifts_are_the_reversed_left_shift():
    """Independent of the ARMv8 model: LSR(a, s) = rev(LSL(rev(a), s)) and
    ASR fills with the sign bit (brute force at width 8)."""
    def rev(x):
        return int(format(x, "08b")[::-1], 2)
    a, s = np.meshgrid(np.arange(256), np.arange(8))
    a, s = a.ravel(), s.ravel()
    lsl = eval_vec(NL.build("LSL", 8), [(a >> i) & 1 for i in range(8)] + [(s >> i) & 1 for i in range(8)])
    lsr = eval_vec(NL.build("LSR", 8), [(a >> i) & 1 for i in range(8)] + [(s >> i) & 1 for i in range(8)])
    asr = eval_vec(NL.build("ASR", 8), [(a >> i) & 1 for i in range(8)] + [(s >> i) & 1 for i in range(8)])
    val = lambda outs: sum(outs[i].astype(np.int64) << i for i in range(8))
    revs = np.array([rev(int(x)) for x in range(256)])
    # LSL on reversed operands, reversed back
    lsl_rev = eval_vec(NL.build("LSL", 8), [(revs[a] >> i) & 1 for i in range(8)] +
                       [(s >> i) & 1 for i in range(8)])
    assert (val(lsr) == revs[val(lsl_rev)]).all()
    sign = (a >> 7) & 1
    fill = np.where(sign == 1, (0xFF << (8 - s)) & 0xFF, 0)
    assert (val(asr) == (val(lsr) | fill)).all()
    assert (val(lsl) == (a << s) & 0xFF).all()


def test_flag_setting_flags_by_brute_force():
    """ADDS/SUBS flags at width 8 from their definitions on signed and
    unsigned integers (independent of the ARMv8 model)."""
    a, b = np.meshgrid(np.arange(256), np.arange(256))
    a, b = a.ravel(), b.ravel()
    sgn = lambda x: np.where(x >= 128, x - 256, x)
    ins = [(a >> i) & 1 for i in range(8)] + [(b >> i) & 1 for i in range(8)]
    for unit, r_u, r_s, carry in (("ADDS", a + b, sgn(a) + sgn(b), a + b > 255),
                                  ("SUBS", a - b, sgn(a) - sgn(b), a >= b)):
        outs = eval_vec(NL.build(unit, 8), ins)
        r = r_u & 255
        assert (sum(outs[i].astype(np.int64) << i for i in range(8)) == r).all()
        assert (outs[8] == (r >> 7)).all()                       # N
        assert (outs[9] == (r == 0)).all()                       # Z
        assert (outs[10] == carry).all()                         # C
        assert (outs[11] == ((r_s < -128) | (r_s > 127))).all()  # V


def test_right_shift_structure():
    for unit in ("LSR", "ASR"):
        for w, stages in ((16, 4), (32, 5)):
            net = NL.build(unit, w)
            # §5: log2(w) MUX stages of w MUXes (4 stages for 16 bits, 5 for 32)
            assert net.depth == stages and len(net.gates) == stages * w
            assert net.bootstraps == 2 * stages * w


@pytest.mark.parametrize("cond", range(14))
def test_csel_all_conditions(cond):
    rng = np.random.default_rng(cond)
    n = 512
    check_unit("CSEL", 8, rng.integers(0, 256, n), rng.integers(0, 256, n), cond,
               np.tile(np.arange(16), n // 16))


def test_structure_matches_the_paper():
    add = NL.build("ADD", 16)
    # §5 "Adder": 16 get_gp (32 gates) + 15/14/12/8 span operators of 3 gates
    # + 15 sum XORs (bit 0 is p_0).  The paper runs 4 carry levels of 2
    # gate levels each in lock step (depth 10); as-soon-as-possible levels
    # let each span start as soon as its inputs exist (depth 9).
    assert len(add.gates) == 32 + 3 * (15 + 14 + 12 + 8) + 15
    assert add.depth == 9
    lsl = NL.build("LSL", 16)
    # §5 "Shifter": 4 stages x 16 MUX
    assert len(lsl.gates) == 64 and lsl.depth == 4 and lsl.bootstraps == 128
    mul = NL.build("MUL", 16)
    assert sum(1 for g in mul.gates if g[5] == 1) == 136      # partial products
    cmp_ = NL.build("CMP", 16)
    sub = NL.build("SUB", 16)
    # §6: Z by a 15-OR tree, V by 5 gates
    assert len(cmp_.gates) == len(sub.gates) + 15 + 5
    # §5 "Signed multiplication": all w^2 partial products at level 1, of
    # which exactly 2(w-1) enter negated (the rows the sign extension made
    # negative), and a full 2w-bit product
    for unit, negated in (("SMULL", 30), ("UMULL", 0)):
        m = NL.build(unit, 16)
        pp = [g[4] for g in m.gates if g[5] == 1]
        assert len(pp) == 256 and len(m.outputs) == 32
        uses = [r for g in m.gates for r in (g[1], g[2], g[3]) if r[0] in set(pp)]
        assert len({r[0] for r in uses if r[1]}) == negated, unit


@pytest.fixture(scope="module")
def lib():
    from paper_2101_03403_gb300 import build
    build.build()
    import paper_2101_03403_gb300 as ce
    return ce


@pytest.mark.parametrize("unit", UNITS + ["CSEL"])
@pytest.mark.parametrize("w", [8, 16, 32])
def test_library_netlist_equals_oracle(lib, unit, w):
    conds = range(14) if unit == "CSEL" else [0]
    for cond in conds:
        mine = NL.build(unit, w, cond)
        theirs = lib.ce_unit_netlist(unit, cond, w)
        assert theirs["n_inputs"] == mine.n_inputs
        assert theirs["depth"] == mine.depth
        assert theirs["gates"] == mine.by_level(), (unit, w, cond)
        assert theirs["outputs"] == list(mine.outputs)
        info = lib.ce_unit_info(unit, cond, w)
        assert info["n_bootstraps"] == mine.bootstraps


@pytest.mark.parametrize("w", [8, 16, 32])
def test_mux_carry_adders_keep_the_bootstraps_in_fewer_levels(w):
    """ADD_MUX / SUB_MUX: the same (g, p) stage, span distances and sums as
    ADD / SUB, each span's carry one MUX (two bootstraps) in place of the
    AND + OR pair: equal bootstrap counts, one level per span, so depth
    1 + log2(w) + 1."""
    import math
    for fast, base in (("ADD_MUX", "ADD"), ("SUB_MUX", "SUB")):
        f, b = NL.build(fast, w), NL.build(base, w)
        assert f.bootstraps == b.bootstraps
        spans = sum(w - d for d in (1 << k for k in range(int(math.log2(w)))))
        assert sum(1 for g in f.gates if g[0] == NL.MUX) == spans
        assert f.depth == 2 + int(math.log2(w))
        assert b.depth > f.depth


def test_tree_multiplier_structure():
    """MUL_TREE: the array multiplier's partial products, compressed by full
    and half adders until every weight holds at most two bits, then one
    MUX-carry prefix adder: far fewer levels than the array (whose rows are
    sequential), at the cost of more bootstraps; the stage count follows the
    Wallace bound for the tallest column (w bits at weight w - 1)."""
    for w, depth in ((8, 13), (16, 18), (32, 22)):
        tree, array = NL.build("MUL_TREE", w), NL.build("MUL", w)
        assert tree.depth == depth and array.depth == 2 * w - 2
        assert tree.bootstraps > array.bootstraps
        ands = [g for g in tree.gates if g[0] == NL.OPS["AND"] and g[5] == 1]
        assert len(ands) == w * (w + 1) // 2          # the partial products, level 1
