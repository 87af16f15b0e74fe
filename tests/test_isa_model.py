"""The plaintext model of the emulated machine's register instructions
(oracle/netlists.py armv8_insn; §4 "Data Processing", §5 "Bitwise
operations" and "Data movement") against independent definitions: per-bit
loops for the bit-field instructions, string reversal for RBIT, byte
arithmetic for REV, Python operators for the rest, exhaustively over the
immediates on random registers."""
import numpy as np

from oracle import netlists as NL

M = 0xFFFF


def bfi_loop(rd, rn, lsb, width):
    out = rd
    for j in range(16):
        if lsb <= j < lsb + width:
            bit = (rn >> (j - lsb)) & 1
            out = (out & ~(1 << j)) | (bit << j)
    return out & M


def test_bitfield_and_reversal_instructions():
    rng = np.random.default_rng(7)
    for _ in range(40):
        rd, rn = (int(x) for x in rng.integers(0, 1 << 16, 2))
        for imm in range(256):
            lsb, width = imm & 15, (imm >> 4) + 1
            assert NL.armv8_insn("BFI", rd, rn, 0, imm, 0, 0)[0] == bfi_loop(rd, rn, lsb, width)
            assert NL.armv8_insn("BFC", rd, rn, 0, imm, 0, 0)[0] == bfi_loop(rd, 0, lsb, width)
        assert NL.armv8_insn("RBIT", rd, rn, 0, 0, 0, 0)[0] == int(format(rn, "016b")[::-1], 2)
        assert NL.armv8_insn("REV", rd, rn, 0, 0, 0, 0)[0] == ((rn & 0xFF) << 8) | (rn >> 8)


def test_immediate_and_negation_instructions():
    rng = np.random.default_rng(8)
    for rn in (int(x) for x in rng.integers(0, 1 << 16, 50)):
        assert NL.armv8_insn("MVN", 0, rn, 0, 0, 0, 0)[0] == (~rn) & M
        for imm in range(256):
            assert NL.armv8_insn("AND_IMM", 0, rn, 0, imm, 0, 0)[0] == rn & imm
            assert NL.armv8_insn("ORR_IMM", 0, rn, 0, imm, 0, 0)[0] == rn | imm
            assert NL.armv8_insn("EOR_IMM", 0, rn, 0, imm, 0, 0)[0] == rn ^ imm
            assert NL.armv8_insn("MOV_IMM", 0, rn, 0, imm, 0, 0)[0] == imm
        for sh in range(40):
            s = sh % 16
            assert NL.armv8_insn("LSL_IMM", 0, rn, 0, sh, 0, 0)[0] == (rn << s) & M
            assert NL.armv8_insn("LSR_IMM", 0, rn, 0, sh, 0, 0)[0] == rn >> s
            signed = rn - (1 << 16) if rn >> 15 else rn
            assert NL.armv8_insn("ASR_IMM", 0, rn, 0, sh, 0, 0)[0] == (signed >> s) & M


def test_register_instructions_and_flags():
    rng = np.random.default_rng(9)
    for _ in range(200):
        rn, rm = (int(x) for x in rng.integers(0, 1 << 16, 2))
        assert NL.armv8_insn("EOR", 0, rn, rm, 0, 0, 0)[0] == rn ^ rm
        assert NL.armv8_insn("ORN", 0, rn, rm, 0, 0, 0)[0] == (rn | ~rm) & M
        assert NL.armv8_insn("ADD", 0, rn, rm, 0, 0, 0)[0] == (rn + rm) & M
        _, f = NL.armv8_insn("CMP", 5, rn, rm, 0, 0, 0)
        N, Z, C, V = f & 1, f >> 1 & 1, f >> 2 & 1, f >> 3 & 1
        r = (rn - rm) & M
        assert (N, Z, C) == (r >> 15, int(r == 0), int(rn >= rm))
        sa, sb = rn - (rn >> 15 << 16), rm - (rm >> 15 << 16)
        assert V == int(not -32768 <= sa - sb <= 32767)


def test_high_half_multiplies():
    """SMULH / UMULH: the high 16 bits of the 32-bit product, against the
    product of the operands read as signed (two's complement) or unsigned
    integers, including the corner cases of the signed range."""
    rng = np.random.default_rng(10)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, 1 << 16, (300, 2))]
    pairs += [(0x8000, 0x8000), (0x8000, 0x7FFF), (0xFFFF, 0xFFFF), (0xFFFF, 1), (0, 0x8000)]
    for rn, rm in pairs:
        sa = rn - 65536 if rn >= 32768 else rn
        sb = rm - 65536 if rm >= 32768 else rm
        p = sa * sb
        assert NL.armv8_insn("SMULH", 0, rn, rm, 0, 0, 0)[0] == (p // 65536) % 65536
        assert NL.armv8_insn("UMULH", 0, rn, rm, 0, 0, 0)[0] == (rn * rm) // 65536
        assert NL.armv8("SMULL", rn, rm, 16) == p % (1 << 32)
