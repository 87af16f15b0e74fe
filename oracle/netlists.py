"""Oracle construction of CryptoEmu's functional units as gate netlists.

TEST INFRASTRUCTURE ONLY (see oracle.py).  Written from the paper's unit
descriptions — §5 "Adder" (three-stage parallel-prefix adder, the span
operator of Stage 2, Kogge-Stone levels of 15/14/12/8 operators for 16 bits),
§5 "Subtractor" (a + NOT b + 1, the extra OR at bit 0), §5 "Shifter" (barrel
shifter of log2(w) MUX stages; the right shifts as the same barrel with the
bit order of input and output reversed, the arithmetic one shifting in the
MSB), §5 "Multiplier" (read as an array multiplier
keeping the low w bits), §5 "Divider" (non-restoring division, add/subtract
chosen by the sign of the partial remainder), §5 "Bitwise operations",
§6 "Conditional Flags" (N, Z by an OR tree, C, V by the formula given there)
— in plain Python, independently of the CUDA library.  Gates are recorded in
creation order with their as-soon-as-possible level; a wire reference is a
pair (wire, negated) and wire -1 is the constant false.

Also: the ARMv8 reference semantics of each unit and a plaintext evaluator.
"""
from __future__ import annotations

from dataclasses import dataclass, field

FALSE = (-1, False)
TRUE = (-1, True)
MUX = 10
OPS = {"NAND": 0, "AND": 1, "OR": 2, "XOR": 3, "NOR": 4, "XNOR": 5, "ANDNY": 6, "ANDYN": 7,
       "ORNY": 8, "ORYN": 9}
UNITS = ["ADD", "ADD_RIPPLE", "SUB", "AND", "ORR", "LSL", "MUL", "UDIV", "CMP", "CSEL", "LSR",
         "ASR", "EOR", "ORN", "ADDS", "SUBS", "SMULL", "UMULL", "ADD_MUX", "SUB_MUX", "MUL_TREE",
         "UDIV_MUX"]
CONDS = ["EQ", "NE", "CS", "CC", "MI", "PL", "VS", "VC", "HI", "LS", "GE", "LT", "GT", "LE"]


def neg(r):
    return (r[0], not r[1])


@dataclass
class Net:
    n_inputs: int
    levels: list = field(default_factory=list)     # level of every wire
    gates: list = field(default_factory=list)      # (op, a, b, c, out, level)
    outputs: list = field(default_factory=list)

    def __post_init__(self):
        self.levels = [0] * self.n_inputs

    def inp(self, i):
        return (i, False)

    def _lvl(self, r):
        return 0 if r[0] < 0 else self.levels[r[0]]

    def g(self, op, a, b):
        lv = 1 + max(self._lvl(a), self._lvl(b))
        out = len(self.levels)
        self.levels.append(lv)
        self.gates.append((OPS[op], a, b, FALSE, out, lv))
        return (out, False)

    def mux(self, s, x, y):
        """s ? x : y (two bootstraps)."""
        lv = 1 + max(self._lvl(s), self._lvl(x), self._lvl(y))
        out = len(self.levels)
        self.levels.append(lv)
        self.gates.append((MUX, s, x, y, out, lv))
        return (out, False)

    def by_level(self):
        """Gates ordered by level, creation order within a level."""
        return sorted(self.gates, key=lambda t: t[5])  # sorted() is stable

    @property
    def depth(self):
        return max((t[5] for t in self.gates), default=0)

    @property
    def bootstraps(self):
        return sum(2 if t[0] == MUX else 1 for t in self.gates)


# --------------------------------------------------------------- adders ---
def prefix_adder(net, a, b, carry_in=None, mux_carry=False):
    """§5 "Adder": stage 1 (g, p) per bit; stage 2 Kogge-Stone combines at
    distances 1, 2, 4, ...; stage 3 sums.  carry_in: None (0), "one" (the
    subtractor's constant 1) or an encrypted wire.  mux_carry: the combined
    G of a span is MUX(P_i; G_{i-d}, G_i) — a span whose bits all propagate
    generates nothing itself, so this equals G_i OR (P_i AND G_{i-d}) — built
    before the AND of the P's; an encrypted carry-in c gives G_0 =
    MUX(p_0; c, g_0) likewise."""
    w = len(a)
    gen, prop = [], []
    for i in range(w):
        gen.append(net.g("AND", a[i], b[i]))
        prop.append(net.g("XOR", a[i], b[i]))
    G, P = list(gen), list(prop)
    if carry_in == "one":
        G[0] = net.g("OR", gen[0], prop[0])
    elif carry_in is not None and mux_carry:
        G[0] = net.mux(prop[0], carry_in, gen[0])
    elif carry_in is not None:
        t = net.g("AND", prop[0], carry_in)
        G[0] = net.g("OR", gen[0], t)
    d = 1
    while d < w:
        G2, P2 = list(G), list(P)
        for i in range(d, w):
            # (G_i, P_i) <- (G_i, P_i) (.) (G_{i-d}, P_{i-d})
            if mux_carry:
                G2[i] = net.mux(P[i], G[i - d], G[i])
                P2[i] = net.g("AND", P[i], P[i - d])
            else:
                t = net.g("AND", P[i], G[i - d])
                P2[i] = net.g("AND", P[i], P[i - d])
                G2[i] = net.g("OR", G[i], t)
        G, P = G2, P2
        d *= 2
    if carry_in is None:
        s0 = prop[0]
    elif carry_in == "one":
        s0 = neg(prop[0])
    else:
        s0 = net.g("XOR", prop[0], carry_in)
    sums = [s0] + [net.g("XOR", prop[i], G[i - 1]) for i in range(1, w)]
    return sums, G[w - 1]


def tree_multiplier(net, a, b):
    """Low w bits of a * b by column compression: the partial products
    a_j AND b_i (i + j < w; i outer) fill one heap per weight; while a heap
    holds more than two bits, each stage replaces, per weight from the
    lowest, every three bits x, y, z by a full adder (u = x XOR y, sum
    u XOR z, carry MUX(u; z, x) one weight up) and a remaining pair of a
    heap taller than two by a half adder (XOR, AND), passing the rest on;
    a new heap receives the carries from below first, then its sums, then
    its passed bits; carries out of the top weight are dropped.  From the
    lowest weight holding two bits up, the two rows are added by the
    MUX-carry prefix adder (a missing second bit is the constant false)."""
    w = len(a)
    heaps = [[] for _ in range(w)]
    for i in range(w):
        for j in range(w - i):
            heaps[i + j].append(net.g("AND", a[j], b[i]))
    while max(len(h) for h in heaps) > 2:
        new = [[] for _ in range(w)]
        for k, h in enumerate(heaps):
            t = 0
            while len(h) - t >= 3:
                x, y, z = h[t:t + 3]
                t += 3
                u = net.g("XOR", x, y)
                new[k].append(net.g("XOR", u, z))
                if k + 1 < w:
                    new[k + 1].append(net.mux(u, z, x))
            if len(h) - t == 2 and len(h) > 2:
                x, y = h[t:t + 2]
                t += 2
                new[k].append(net.g("XOR", x, y))
                if k + 1 < w:
                    new[k + 1].append(net.g("AND", x, y))
            new[k].extend(h[t:])
        heaps = new
    two = [k for k in range(w) if len(heaps[k]) == 2]
    if not two:
        return [h[0] for h in heaps]
    k0 = two[0]
    x = [heaps[k][0] for k in range(k0, w)]
    y = [heaps[k][1] if len(heaps[k]) == 2 else FALSE for k in range(k0, w)]
    sums, _ = prefix_adder(net, x, y, mux_carry=True)
    return [heaps[k][0] for k in range(k0)] + sums


def ripple_adder(net, a, b):
    w = len(a)
    gen, prop = [], []
    for i in range(w):
        gen.append(net.g("AND", a[i], b[i]))
        prop.append(net.g("XOR", a[i], b[i]))
    out = [prop[0]]
    carry = gen[0]
    for i in range(1, w):
        out.append(net.g("XOR", prop[i], carry))
        if i < w - 1:
            t = net.g("AND", prop[i], carry)
            carry = net.g("OR", gen[i], t)
    return out


def or_reduce(net, xs):
    xs = list(xs)
    while len(xs) > 1:
        nxt = [net.g("OR", xs[i], xs[i + 1]) for i in range(0, len(xs) - 1, 2)]
        if len(xs) % 2:
            nxt.append(xs[-1])
        xs = nxt
    return xs[0]


def cond_bit(net, cond, N, Z, C, V):
    name = CONDS[cond]
    if name == "EQ": return Z
    if name == "NE": return neg(Z)
    if name == "CS": return C
    if name == "CC": return neg(C)
    if name == "MI": return N
    if name == "PL": return neg(N)
    if name == "VS": return V
    if name == "VC": return neg(V)
    if name == "HI": return net.g("ANDYN", C, Z)
    if name == "LS": return neg(net.g("ANDYN", C, Z))
    if name == "GE": return net.g("XNOR", N, V)
    if name == "LT": return net.g("XOR", N, V)
    t = net.g("XNOR", N, V)
    gt = net.g("ANDNY", Z, t)
    return gt if name == "GT" else neg(gt)


def full_product(net, a, b, signed):
    """§5 "Signed multiplication" / "Unsigned multiplication": the whole
    2w-bit product.  Signed operands: a * b = sum over i, j < w-1 of
    a_j b_i 2^(i+j) + a_{w-1} b_{w-1} 2^(2w-2) - (sum over j < w-1 of
    a_j b_{w-1} 2^(j+w-1) + the same with a, b swapped); each negative row
    -x 2^k equals (NOT x - 1) 2^k, so the two rows become negated partial
    products plus the constant -2 (2^(2w-2) - 2^(w-1)) = 2^w - 2^(2w-1), which
    is 2^w + 2^(2w-1) mod 2^(2w): the constant that replaces the sign
    extension.  2^w enters as the carry-in of the final adder and 2^(2w-1)
    flips the top bit.  The partial products are summed row by row with
    their carries kept (carry-save), then the high half by the prefix adder."""
    w = len(a)
    pp = []
    for i in range(w):
        row = []
        for j in range(w):
            x = net.g("AND", a[j], b[i])
            row.append(neg(x) if signed and ((i == w - 1) != (j == w - 1)) else x)
        pp.append(row)
    S = {j: pp[0][j] for j in range(w)}
    C = {}
    for i in range(1, w):
        nxt = {}
        for k in range(i, i + w):
            y = pp[i][k - i]
            have = [v for v in (S.get(k), C.get(k)) if v is not None]
            if not have:
                S[k] = y
            elif len(have) == 1:
                x = have[0]
                S[k] = net.g("XOR", x, y)
                nxt[k + 1] = net.g("AND", x, y)
            else:
                x, c = S[k], C[k]
                u = net.g("XOR", x, y)
                S[k] = net.g("XOR", u, c)
                nxt[k + 1] = net.mux(u, c, x)      # carry = majority(x, y, c)
        C = nxt
    # nothing reaches weight 2w-1 but the carry out of weights w..2w-2
    hx = [S.get(w + k, FALSE) for k in range(w - 1)]
    hy = [C.get(w + k, FALSE) for k in range(w - 1)]
    hi, top = prefix_adder(net, hx, hy, "one" if signed else None)
    return [S[k] for k in range(w)] + hi + [neg(top) if signed else top]


def build(unit: str, w: int = 16, cond: int = 0) -> Net:
    net = Net(2 * w + (4 if unit == "CSEL" else 0))
    a = [net.inp(i) for i in range(w)]
    b = [net.inp(w + i) for i in range(w)]
    if unit == "ADD":
        out, _ = prefix_adder(net, a, b)
    elif unit == "ADD_RIPPLE":
        out = ripple_adder(net, a, b)
    elif unit == "SUB":
        out, _ = prefix_adder(net, a, [neg(x) for x in b], "one")
    elif unit == "ADD_MUX":
        out, _ = prefix_adder(net, a, b, mux_carry=True)
    elif unit == "SUB_MUX":
        out, _ = prefix_adder(net, a, [neg(x) for x in b], "one", mux_carry=True)
    elif unit in ("AND", "ORR"):
        out = [net.g("AND" if unit == "AND" else "OR", a[i], b[i]) for i in range(w)]
    elif unit == "EOR":
        out = [net.g("XOR", a[i], b[i]) for i in range(w)]
    elif unit == "ORN":                     # a OR NOT b: the ORYN gate per bit
        out = [net.g("ORYN", a[i], b[i]) for i in range(w)]
    elif unit == "LSL":
        x, k, sh = list(a), 0, 1
        while sh < w:
            x = [net.mux(b[k], x[j - sh] if j >= sh else FALSE, x[j]) for j in range(w)]
            k += 1
            sh *= 2
        out = x
    elif unit in ("LSR", "ASR"):
        # §5 "Logic right shift/Arithmetic right shift": the LSL barrel on
        # the bit-reversed operand, output reversed back; ARS fills with the
        # MSB instead of zero.
        fill = a[w - 1] if unit == "ASR" else FALSE
        x, k, sh = list(reversed(a)), 0, 1
        while sh < w:
            x = [net.mux(b[k], x[j - sh] if j >= sh else fill, x[j]) for j in range(w)]
            k += 1
            sh *= 2
        out = list(reversed(x))
    elif unit == "MUL":
        pp = [[net.g("AND", a[j], b[i]) for j in range(w - i)] for i in range(w)]
        S = list(pp[0])
        carries = {}
        for i in range(1, w):
            nxt = {}
            for k in range(i, w):
                x, y = S[k], pp[i][k - i]
                top = k + 1 == w
                if k not in carries:            # half adder
                    s = net.g("XOR", x, y)
                    if not top:
                        nxt[k + 1] = net.g("AND", x, y)
                else:                           # full adder, carry = MAJ via MUX
                    u = net.g("XOR", x, y)
                    s = net.g("XOR", u, carries[k])
                    if not top:
                        nxt[k + 1] = net.mux(u, carries[k], x)
                S[k] = s
            carries = nxt
        out = S
    elif unit == "MUL_TREE":
        out = tree_multiplier(net, a, b)
    elif unit in ("UDIV", "UDIV_MUX"):
        A = [FALSE] * (w + 1)
        Q = list(a)
        for _ in range(w):
            sign = A[w]
            shifted = [Q[w - 1]] + A[:w]          # [A, Q] << 1, old A_w dropped
            Q = [None] + Q[:w - 1]
            sub = neg(sign)                        # subtract while A >= 0
            dx = [net.g("XOR", b[k], sub) for k in range(w)] + [sub]
            A, _ = prefix_adder(net, shifted, dx, sub, mux_carry=unit == "UDIV_MUX")
            Q[0] = neg(A[w])
        nonzero = or_reduce(net, b)
        out = [net.g("AND", Q[k], nonzero) for k in range(w)]
    elif unit in ("CMP", "SUBS"):
        s, carry = prefix_adder(net, a, [neg(x) for x in b], "one")
        N = s[w - 1]
        Z = neg(or_reduce(net, s))
        x1 = net.g("ANDNY", a[w - 1], b[w - 1])
        x2 = net.g("AND", x1, s[w - 1])
        y1 = net.g("ANDYN", a[w - 1], b[w - 1])
        y2 = net.g("ANDYN", y1, s[w - 1])
        V = net.g("OR", x2, y2)
        out = ([] if unit == "CMP" else s) + [N, Z, carry, V]
    elif unit == "ADDS":
        # §6's flags on a + b: V = (!a !b s) + (a b !s) with the operands as given
        s, carry = prefix_adder(net, a, b)
        N = s[w - 1]
        Z = neg(or_reduce(net, s))
        x1 = net.g("NOR", a[w - 1], b[w - 1])
        x2 = net.g("AND", x1, s[w - 1])
        y1 = net.g("AND", a[w - 1], b[w - 1])
        y2 = net.g("ANDYN", y1, s[w - 1])
        V = net.g("OR", x2, y2)
        out = s + [N, Z, carry, V]
    elif unit in ("SMULL", "UMULL"):
        out = full_product(net, a, b, unit == "SMULL")
    elif unit == "CSEL":
        N, Z, C, V = (net.inp(2 * w + i) for i in range(4))
        c = cond_bit(net, cond, N, Z, C, V)
        out = [net.mux(c, a[j], b[j]) for j in range(w)]
    else:
        raise ValueError(unit)
    net.outputs = out
    return net


# -------------------------------------------------------------- evaluate ---
GATE_FN = {
    0: lambda x, y: 1 - (x & y), 1: lambda x, y: x & y, 2: lambda x, y: x | y,
    3: lambda x, y: x ^ y, 4: lambda x, y: 1 - (x | y), 5: lambda x, y: 1 - (x ^ y),
    6: lambda x, y: (1 - x) & y, 7: lambda x, y: x & (1 - y), 8: lambda x, y: (1 - x) | y,
    9: lambda x, y: x | (1 - y),
}


def eval_plain(net: Net, inputs: list[int]) -> list[int]:
    """Evaluate on plaintext bits, gate by gate in level order."""
    val = list(inputs) + [None] * (len(net.levels) - net.n_inputs)

    def rd(r):
        v = 0 if r[0] < 0 else val[r[0]]
        return 1 - v if r[1] else v

    for op, a, b, c, out, _ in net.by_level():
        val[out] = (rd(b) if rd(a) else rd(c)) if op == MUX else GATE_FN[op](rd(a), rd(b))
    return [rd(r) for r in net.outputs]


def bits(x: int, w: int) -> list[int]:
    return [(x >> i) & 1 for i in range(w)]


def from_bits(bs) -> int:
    return sum(b << i for i, b in enumerate(bs))


def armv8(unit: str, a: int, b: int, w: int = 16, cond: int = 0, nzcv: int = 0):
    """ARMv8 semantics truncated to w bits.  CMP returns [N, Z, C, V];
    CSEL takes nzcv as bits N|Z<<1|C<<2|V<<3."""
    m = (1 << w) - 1
    if unit in ("ADD", "ADD_RIPPLE", "ADD_MUX"):
        return (a + b) & m
    if unit in ("SUB", "SUB_MUX"):
        return (a - b) & m
    if unit == "AND":
        return a & b
    if unit == "ORR":
        return a | b
    if unit == "EOR":
        return a ^ b
    if unit == "ORN":
        return (a | ~b) & m
    if unit == "LSL":
        return (a << (b % w)) & m
    if unit == "LSR":
        return a >> (b % w)
    if unit == "ASR":
        sa = a - (1 << w) if a >> (w - 1) else a
        return (sa >> (b % w)) & m
    if unit in ("MUL", "MUL_TREE"):
        return (a * b) & m
    if unit == "UMULL":
        return a * b
    if unit == "SMULL":
        sa = a - (1 << w) if a >> (w - 1) else a
        sb = b - (1 << w) if b >> (w - 1) else b
        return (sa * sb) & ((1 << 2 * w) - 1)
    if unit in ("UDIV", "UDIV_MUX"):
        return 0 if b == 0 else a // b
    if unit == "CMP":
        r = (a - b) & m
        sa, sb, sr = a >> (w - 1), b >> (w - 1), r >> (w - 1)
        return [sr, int(r == 0), int(a >= b), int(sa != sb and sr != sa)]
    if unit == "SUBS":
        return [(a - b) & m] + armv8("CMP", a, b, w)
    if unit == "ADDS":
        r = (a + b) & m
        sa, sb, sr = a >> (w - 1), b >> (w - 1), r >> (w - 1)
        return [r, sr, int(r == 0), int(a + b > m), int(sa == sb and sr != sa)]
    if unit == "CSEL":
        N, Z, C, V = (nzcv >> i & 1 for i in range(4))
        table = {"EQ": Z, "NE": 1 - Z, "CS": C, "CC": 1 - C, "MI": N, "PL": 1 - N, "VS": V,
                 "VC": 1 - V, "HI": C & (1 - Z), "LS": 1 - (C & (1 - Z)), "GE": int(N == V),
                 "LT": int(N != V), "GT": (1 - Z) & int(N == V), "LE": 1 - ((1 - Z) & int(N == V))}
        return a if table[CONDS[cond]] else b
    raise ValueError(unit)


def armv8_insn(op: str, rd: int, rn: int, rm: int, imm: int, cond: int, nzcv: int,
               w: int = 16):
    """One register instruction of the emulated machine on plaintext values:
    returns (new rd value, new nzcv).  §4 "Data Processing" and §5/§6 units;
    imm is the 8-bit instruction immediate; BFC/BFI take lsb = imm & 15 and
    width = (imm >> 4) + 1 (clipped at the register's top bit)."""
    m = (1 << w) - 1
    if op == "CMP":
        N, Z, C, V = armv8("CMP", rn, rm, w)
        return rd, N | Z << 1 | C << 2 | V << 3
    if op == "CSEL":
        return armv8("CSEL", rn, rm, w, cond, nzcv), nzcv
    if op in ("ADDS", "SUBS"):
        r, N, Z, C, V = armv8(op, rn, rm, w)
        return r, N | Z << 1 | C << 2 | V << 3
    if op == "MOV":
        return rn, nzcv
    if op == "MOV_IMM":
        return imm, nzcv
    if op == "SMULH":
        return armv8("SMULL", rn, rm, w) >> w, nzcv
    if op == "UMULH":
        return armv8("UMULL", rn, rm, w) >> w, nzcv
    if op in ("LSL_IMM", "LSR_IMM", "ASR_IMM"):
        return armv8(op[:3], rn, imm % w, w), nzcv
    if op == "MVN":
        return ~rn & m, nzcv
    if op in ("AND_IMM", "ORR_IMM", "EOR_IMM"):
        return armv8(op[:3], rn, imm, w), nzcv
    lsb, width = imm & 15, (imm >> 4) + 1
    field = ((1 << width) - 1) << lsb & m
    if op == "BFC":
        return rd & ~field & m, nzcv
    if op == "BFI":
        return (rd & ~field | (rn << lsb) & field) & m, nzcv
    if op == "RBIT":
        return from_bits(bits(rn, w)[::-1]), nzcv
    if op == "REV":
        return from_bits(sum((bits(rn, w)[8 * k:8 * k + 8] for k in reversed(range(w // 8))), [])), nzcv
    return armv8(op, rn, rm, w), nzcv


def eval_ciphertext(keys, net: Net, inputs):
    """Evaluate on ciphertexts with the oracle's gates, level by level."""
    from . import oracle as O
    p = keys.params
    fals = O.constant(p, 0)
    val = list(inputs) + [None] * (len(net.levels) - net.n_inputs)

    def rd(r):
        v = fals if r[0] < 0 else val[r[0]]
        return O.not_(p, v) if r[1] else v

    for depth in range(1, net.depth + 1):
        lvl = [t for t in net.gates if t[5] == depth]
        plain = [t for t in lvl if t[0] != MUX]
        if plain:
            outs = O.gates(keys, [t[0] for t in plain], [rd(t[1]) for t in plain],
                           [rd(t[2]) for t in plain])
            for t, o in zip(plain, outs):
                val[t[4]] = o
        muxes = [t for t in lvl if t[0] == MUX]
        if muxes:
            outs = O.muxes(keys, [rd(t[1]) for t in muxes], [rd(t[2]) for t in muxes],
                           [rd(t[3]) for t in muxes])
            for t, o in zip(muxes, outs):
                val[t[4]] = o
    return [rd(r) for r in net.outputs]
