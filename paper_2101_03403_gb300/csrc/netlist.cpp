// Functional-unit netlists over bootstrapped gates (§5 "Data Processing
// Units", §6 "Conditional Flags").  Gates are created in a fixed order; the
// finished netlist lists them by level, creation order within a level.
#include "netlist.h"

#include <algorithm>

namespace ce {

namespace {

enum : uint8_t { NAND = 0, AND = 1, OR = 2, XOR = 3, NOR = 4, XNOR = 5, ANDNY = 6, ANDYN = 7,
                 ORNY = 8, ORYN = 9 };

class Builder {
 public:
  explicit Builder(int n_inputs) : n_inputs_(n_inputs), level_(n_inputs, 0) {}
  Ref in(int i) const { return Ref{i, false}; }
  Ref gate(uint8_t op, Ref a, Ref b) { return add(op, a, b, Ref{}); }
  // s ? x : y
  Ref mux(Ref s, Ref x, Ref y) { return add(kOpMux, s, x, y); }

  Netlist finish(const std::vector<Ref> &outputs) {
    Netlist n;
    n.n_inputs = n_inputs_;
    n.n_wires = static_cast<int32_t>(level_.size());
    std::vector<NGate> g = gates_;
    std::stable_sort(g.begin(), g.end(),
                     [](const NGate &x, const NGate &y) { return x.level < y.level; });
    n.gates = g;
    int depth = 0;
    for (const auto &x : g) depth = std::max(depth, x.level);
    n.depth = depth;
    n.level_begin.assign(depth + 1, 0);
    size_t k = 0;
    for (int L = 1; L <= depth; ++L) {
      n.level_begin[L - 1] = static_cast<int32_t>(k);
      while (k < g.size() && g[k].level == L) ++k;
    }
    n.level_begin[depth] = static_cast<int32_t>(g.size());
    n.outputs = outputs;
    return n;
  }

 private:
  int lvl(Ref r) const { return r.wire < 0 ? 0 : level_[r.wire]; }
  Ref add(uint8_t op, Ref a, Ref b, Ref c) {
    const int L = 1 + std::max({lvl(a), lvl(b), op == kOpMux ? lvl(c) : 0});
    const int32_t w = static_cast<int32_t>(level_.size());
    level_.push_back(L);
    gates_.push_back(NGate{op, a, b, c, w, L});
    return Ref{w, false};
  }
  int n_inputs_;
  std::vector<int> level_;
  std::vector<NGate> gates_;
};

struct AdderOut {
  std::vector<Ref> sum;
  Ref carry;
};

// Parallel-prefix adder (§5 "Adder"): stage 1 g_i = a_i AND b_i,
// p_i = a_i XOR b_i; stage 2 Kogge-Stone span combines at distances 1, 2,
// 4, ...: (G_i, P_i) <- (G_i OR (P_i AND G_{i-d}), P_i AND P_{i-d}) for
// i >= d (created as the AND for G, the AND for P, then the OR); stage 3
// s_i = p_i XOR G_{i-1}.  Carry-in: constant 1 folds into bit 0 as
// G_0 = g_0 OR p_0 and s_0 = NOT p_0 (§5 "Subtractor"); an encrypted
// carry-in c gives G_0 = g_0 OR (p_0 AND c) and s_0 = p_0 XOR c.
// mux_prefix: the span combine's G as one MUX, G_i <- P_i ? G_{i-d} : G_i
// (equal to G_i OR (P_i AND G_{i-d}) because a span that propagates
// generates nothing of its own), created before P's AND: the same
// bootstraps in one level per span instead of two; likewise an encrypted
// carry-in folds in as G_0 = p_0 ? c : g_0.
AdderOut kogge_stone(Builder &B, const std::vector<Ref> &a, const std::vector<Ref> &b,
                     int cin_kind, Ref cin, bool mux_prefix = false) {
  const int w = static_cast<int>(a.size());
  std::vector<Ref> g(w), p(w);
  for (int i = 0; i < w; ++i) {
    g[i] = B.gate(AND, a[i], b[i]);
    p[i] = B.gate(XOR, a[i], b[i]);
  }
  std::vector<Ref> G = g, P = p;
  if (cin_kind == 1) {
    G[0] = B.gate(OR, g[0], p[0]);
  } else if (cin_kind == 2 && mux_prefix) {
    G[0] = B.mux(p[0], cin, g[0]);
  } else if (cin_kind == 2) {
    const Ref t = B.gate(AND, p[0], cin);
    G[0] = B.gate(OR, g[0], t);
  }
  for (int d = 1; d < w; d *= 2) {
    std::vector<Ref> nG = G, nP = P;
    for (int i = d; i < w; ++i) {
      if (mux_prefix) {
        nG[i] = B.mux(P[i], G[i - d], G[i]);
        nP[i] = B.gate(AND, P[i], P[i - d]);
      } else {
        const Ref t = B.gate(AND, P[i], G[i - d]);
        nP[i] = B.gate(AND, P[i], P[i - d]);
        nG[i] = B.gate(OR, G[i], t);
      }
    }
    G = nG;
    P = nP;
  }
  AdderOut r;
  r.sum.resize(w);
  if (cin_kind == 0) r.sum[0] = p[0];
  else if (cin_kind == 1) r.sum[0] = !p[0];
  else r.sum[0] = B.gate(XOR, p[0], cin);
  for (int i = 1; i < w; ++i) r.sum[i] = B.gate(XOR, p[i], G[i - 1]);
  r.carry = G[w - 1];
  return r;
}

// Ripple-carry adder: g, p per bit; c_1 = g_0; for i >= 1: s_i = p_i XOR c_i,
// then (below the top bit) c_{i+1} = g_i OR (p_i AND c_i).
std::vector<Ref> ripple(Builder &B, const std::vector<Ref> &a, const std::vector<Ref> &b) {
  const int w = static_cast<int>(a.size());
  std::vector<Ref> g(w), p(w), s(w);
  for (int i = 0; i < w; ++i) {
    g[i] = B.gate(AND, a[i], b[i]);
    p[i] = B.gate(XOR, a[i], b[i]);
  }
  s[0] = p[0];
  Ref c = g[0];
  for (int i = 1; i < w; ++i) {
    s[i] = B.gate(XOR, p[i], c);
    if (i < w - 1) {
      const Ref t = B.gate(AND, p[i], c);
      c = B.gate(OR, g[i], t);
    }
  }
  return s;
}

// OR reduction by pairwise levels (§6: Z flag from an OR tree); an odd last
// element passes to the next level unchanged.
Ref or_tree(Builder &B, std::vector<Ref> x) {
  while (x.size() > 1) {
    std::vector<Ref> y;
    for (size_t i = 0; i + 1 < x.size(); i += 2) y.push_back(B.gate(OR, x[i], x[i + 1]));
    if (x.size() % 2) y.push_back(x.back());
    x = y;
  }
  return x[0];
}

std::vector<Ref> slice(const Builder &B, int from, int w) {
  std::vector<Ref> r(w);
  for (int i = 0; i < w; ++i) r[i] = B.in(from + i);
  return r;
}

// Condition bit of an ARM condition code from (N, Z, C, V).
Ref condition(Builder &B, int cond, Ref N, Ref Z, Ref C, Ref V) {
  switch (cond) {
    case 0: return Z;                        // EQ
    case 1: return !Z;                       // NE
    case 2: return C;                        // CS / HS
    case 3: return !C;                       // CC / LO
    case 4: return N;                        // MI
    case 5: return !N;                       // PL
    case 6: return V;                        // VS
    case 7: return !V;                       // VC
    case 8: return B.gate(ANDYN, C, Z);      // HI: C and not Z
    case 9: return !B.gate(ANDYN, C, Z);     // LS
    case 10: return B.gate(XNOR, N, V);      // GE: N == V
    case 11: return B.gate(XOR, N, V);       // LT
    case 12: {                               // GT: not Z and N == V
      const Ref t = B.gate(XNOR, N, V);
      return B.gate(ANDNY, Z, t);
    }
    default: {                               // LE
      const Ref t = B.gate(XNOR, N, V);
      return !B.gate(ANDNY, Z, t);
    }
  }
}

// Low w bits of a * b by column compression (a Wallace tree).  The partial
// products a_j AND b_i (i + j < w, i outer) go to one heap per weight.  While
// a heap holds more than two bits, a stage walks the weights upward: every
// three bits x, y, z become a full adder (u = x ^ y; sum u ^ z stays; carry
// = u ? z : x, one MUX, moves one weight up) and the last pair of a heap that
// held more than two a half adder (XOR, AND); other bits pass on.  A heap of
// the next stage holds, in order, the carries from the weight below, its own
// sums, then its passed bits; carries out of the top weight are dropped.  The
// two rows left from the lowest weight with two bits up are summed by the
// MUX-carry prefix adder (a missing second bit: constant false).
std::vector<Ref> tree_multiplier(Builder &B, const std::vector<Ref> &a, const std::vector<Ref> &b) {
  const int w = static_cast<int>(a.size());
  std::vector<std::vector<Ref>> heap(w);
  for (int i = 0; i < w; ++i)
    for (int j = 0; j + i < w; ++j) heap[i + j].push_back(B.gate(AND, a[j], b[i]));
  auto tallest = [&] {
    size_t m = 0;
    for (const auto &h : heap) m = std::max(m, h.size());
    return m;
  };
  while (tallest() > 2) {
    std::vector<std::vector<Ref>> next(w);
    for (int k = 0; k < w; ++k) {
      const std::vector<Ref> &h = heap[k];
      size_t t = 0;
      for (; h.size() - t >= 3; t += 3) {
        const Ref u = B.gate(XOR, h[t], h[t + 1]);
        next[k].push_back(B.gate(XOR, u, h[t + 2]));
        if (k + 1 < w) next[k + 1].push_back(B.mux(u, h[t + 2], h[t]));
      }
      if (h.size() - t == 2 && h.size() > 2) {
        next[k].push_back(B.gate(XOR, h[t], h[t + 1]));
        if (k + 1 < w) next[k + 1].push_back(B.gate(AND, h[t], h[t + 1]));
        t += 2;
      }
      for (; t < h.size(); ++t) next[k].push_back(h[t]);
    }
    heap = std::move(next);
  }
  int k0 = 0;
  while (k0 < w && heap[k0].size() < 2) ++k0;
  std::vector<Ref> out(w);
  for (int k = 0; k < k0; ++k) out[k] = heap[k][0];
  if (k0 == w) return out;
  std::vector<Ref> x, y;
  for (int k = k0; k < w; ++k) {
    x.push_back(heap[k][0]);
    y.push_back(heap[k].size() == 2 ? heap[k][1] : constant(false));
  }
  const std::vector<Ref> s = kogge_stone(B, x, y, 0, Ref{}, true).sum;
  for (int k = k0; k < w; ++k) out[k] = s[k - k0];
  return out;
}

// Full-width array multiplier: the 2w-bit product of a and b.  Partial
// products pp[i][j] = a_j AND b_i at weight i + j.  Signed (§5 "Signed
// multiplication": the partial products' sign extension to 2w bits replaced
// by a constant, the Baugh-Wooley form): the bits with exactly one of i, j
// equal to w - 1 enter negated (a free NOT of the AND), and 2^w + 2^(2w-1) is
// added, 2^w as the carry-in of the final adder and 2^(2w-1) as a negation of
// the product's top bit.  Rows 1..w-1 add pp[i] into the running sum at
// weights i..i+w-1 together with the previous row's carries (carry-save: a
// full adder is s = x ^ y ^ c, carry = (x ^ y) ? c : x as one MUX; a cell
// with two inputs is a half adder, with one a wire); bit k < w is final after
// row k, and the high half is the Kogge-Stone sum of the remaining sum and
// carry bits (§5 "Adder").
std::vector<Ref> full_multiplier(Builder &B, const std::vector<Ref> &a, const std::vector<Ref> &b,
                                 bool sign) {
  const int w = static_cast<int>(a.size());
  std::vector<std::vector<Ref>> pp(w, std::vector<Ref>(w));
  for (int i = 0; i < w; ++i)
    for (int j = 0; j < w; ++j) {
      pp[i][j] = B.gate(AND, a[j], b[i]);
      if (sign && ((i == w - 1) != (j == w - 1))) pp[i][j] = !pp[i][j];
    }
  std::vector<Ref> S(2 * w), C(2 * w + 1);
  std::vector<bool> hasS(2 * w, false), hasC(2 * w + 1, false);
  for (int j = 0; j < w; ++j) {
    S[j] = pp[0][j];
    hasS[j] = true;
  }
  for (int i = 1; i < w; ++i) {
    std::vector<Ref> nC(2 * w + 1);
    std::vector<bool> nhas(2 * w + 1, false);
    for (int k = i; k < i + w; ++k) {
      const Ref y = pp[i][k - i];
      if (!hasS[k] && !hasC[k]) {
        S[k] = y;
      } else if (!hasS[k] || !hasC[k]) {
        const Ref x = hasS[k] ? S[k] : C[k];
        S[k] = B.gate(XOR, x, y);
        nC[k + 1] = B.gate(AND, x, y);
        nhas[k + 1] = true;
      } else {
        const Ref x = S[k];
        const Ref u = B.gate(XOR, x, y);
        S[k] = B.gate(XOR, u, C[k]);
        nC[k + 1] = B.mux(u, C[k], x);
        nhas[k + 1] = true;
      }
      hasS[k] = true;
    }
    C = nC;
    hasC = nhas;
  }
  // Weight 2w-1 holds no sum or carry bit (the top cell of every row only
  // passes its partial product on), so the high half is the (w-1)-bit sum of
  // weights w..2w-2 with its carry-out as bit 2w-1.
  std::vector<Ref> hx(w - 1), hy(w - 1);
  for (int k = 0; k + 1 < w; ++k) {
    hx[k] = hasS[w + k] ? S[w + k] : constant(false);
    hy[k] = hasC[w + k] ? C[w + k] : constant(false);
  }
  AdderOut r = kogge_stone(B, hx, hy, sign ? 1 : 0, Ref{});
  std::vector<Ref> hi = r.sum;
  hi.push_back(sign ? !r.carry : r.carry);
  std::vector<Ref> o(S.begin(), S.begin() + w);
  o.insert(o.end(), hi.begin(), hi.end());
  return o;
}

}  // namespace

int32_t Netlist::bootstraps() const {
  int32_t n = 0;
  for (const auto &g : gates) n += g.op == kOpMux ? 2 : 1;
  return n;
}

bool build_unit(int unit, int w, int cond, Netlist *out) {
  if (w < 2 || w > 32 || (w & (w - 1)) || unit < 0 || unit >= kUnitCount) return false;
  if (unit == kUnitCsel && (cond < 0 || cond > 13)) return false;
  const int n_in = unit == kUnitCsel ? 2 * w + 4 : 2 * w;
  Builder B(n_in);
  const std::vector<Ref> a = slice(B, 0, w), b = slice(B, w, w);
  std::vector<Ref> o;
  switch (unit) {
    case kUnitAdd:
      o = kogge_stone(B, a, b, 0, Ref{}).sum;
      break;
    case kUnitAddRipple:
      o = ripple(B, a, b);
      break;
    case kUnitSub: {
      std::vector<Ref> nb(w);
      for (int i = 0; i < w; ++i) nb[i] = !b[i];
      o = kogge_stone(B, a, nb, 1, Ref{}).sum;
      break;
    }
    case kUnitAddMux:
      o = kogge_stone(B, a, b, 0, Ref{}, true).sum;
      break;
    case kUnitMulTree:
      o = tree_multiplier(B, a, b);
      break;
    case kUnitSubMux: {
      std::vector<Ref> nb(w);
      for (int i = 0; i < w; ++i) nb[i] = !b[i];
      o = kogge_stone(B, a, nb, 1, Ref{}, true).sum;
      break;
    }
    case kUnitAnd:
    case kUnitOrr:
    case kUnitEor:
    case kUnitOrn: {
      const uint8_t op = unit == kUnitAnd ? AND : unit == kUnitOrr ? OR : unit == kUnitEor ? XOR : ORYN;
      for (int i = 0; i < w; ++i) o.push_back(B.gate(op, a[i], b[i]));
      break;
    }
    case kUnitLsl: {
      // Barrel shifter: stage k selects, per bit j, x_{j-2^k} (0 below 2^k)
      // when amount bit k is set; amount bits above log2(w) are ignored
      // (shift amount taken mod w).
      std::vector<Ref> x = a;
      for (int k = 0, sh = 1; sh < w; ++k, sh *= 2) {
        std::vector<Ref> y(w);
        for (int j = 0; j < w; ++j) y[j] = B.mux(b[k], j >= sh ? x[j - sh] : constant(false), x[j]);
        x = y;
      }
      o = x;
      break;
    }
    case kUnitLsr:
    case kUnitAsr: {
      // §5: the left-shift barrel on the operand in reversed bit order, the
      // result reversed back; the arithmetic shift brings in the MSB where
      // the logical one brings in zeros.
      const Ref fill = unit == kUnitAsr ? a[w - 1] : constant(false);
      std::vector<Ref> x(a.rbegin(), a.rend());
      for (int k = 0, sh = 1; sh < w; ++k, sh *= 2) {
        std::vector<Ref> y(w);
        for (int j = 0; j < w; ++j) y[j] = B.mux(b[k], j >= sh ? x[j - sh] : fill, x[j]);
        x = y;
      }
      o.assign(x.rbegin(), x.rend());
      break;
    }
    case kUnitMul: {
      // Array multiplier, low w bits: partial products pp[i][j] = a_j AND b_i
      // (i + j < w); row i (i >= 1) adds pp[i] into the running sum at
      // positions k >= i with carries passed to position k+1 of the next
      // row: half adders in row 1, full adders after (s = x ^ y ^ z,
      // carry = MAJ(x, y, z) = (x ^ y) ? z : x); carries out of the top bit
      // are dropped.  Bit i is final after row i.
      std::vector<std::vector<Ref>> pp(w);
      for (int i = 0; i < w; ++i)
        for (int j = 0; j + i < w; ++j) pp[i].push_back(B.gate(AND, a[j], b[i]));
      std::vector<Ref> S = pp[0];
      std::vector<Ref> C(w + 1);
      std::vector<bool> has(w + 1, false);
      for (int i = 1; i < w; ++i) {
        std::vector<Ref> nC(w + 1);
        std::vector<bool> nhas(w + 1, false);
        for (int k = i; k < w; ++k) {
          const Ref x = S[k], y = pp[i][k - i];
          Ref s, carry;
          const bool top = (k + 1 == w);
          if (!has[k]) {
            s = B.gate(XOR, x, y);
            if (!top) carry = B.gate(AND, x, y);
          } else {
            const Ref u = B.gate(XOR, x, y);
            s = B.gate(XOR, u, C[k]);
            if (!top) carry = B.mux(u, C[k], x);
          }
          S[k] = s;
          if (!top) {
            nC[k + 1] = carry;
            nhas[k + 1] = true;
          }
        }
        C = nC;
        has = nhas;
      }
      o = S;
      break;
    }
    case kUnitUdiv:
    case kUnitUdivMux: {
      // Non-restoring division (§5 "Divider") with a (w+1)-bit partial
      // remainder A (two's complement, sign A_w) and D = b extended by a
      // zero bit.  Per iteration: sgn = A_w before the shift; [A, Q] <<= 1;
      // SUB = NOT sgn; A = A + (D XOR SUB) + SUB (the XOR of the constant
      // top bit of D is NOT sgn, free); Q_0 = NOT A_w.  Then ARMv8 UDIV
      // semantics for a zero divisor: Q = Q AND (OR of all divisor bits).
      std::vector<Ref> A(w + 1, constant(false)), Q = a;
      for (int it = 0; it < w; ++it) {
        const Ref sgn = A[w];
        std::vector<Ref> As(w + 1);
        As[0] = Q[w - 1];
        for (int k = 1; k <= w; ++k) As[k] = A[k - 1];
        for (int k = w - 1; k >= 1; --k) Q[k] = Q[k - 1];
        const Ref sub = !sgn;
        std::vector<Ref> Dx(w + 1);
        for (int k = 0; k < w; ++k) Dx[k] = B.gate(XOR, b[k], sub);
        Dx[w] = sub;
        A = kogge_stone(B, As, Dx, 2, sub, unit == kUnitUdivMux).sum;
        Q[0] = !A[w];
      }
      const Ref nz = or_tree(B, b);
      for (int k = 0; k < w; ++k) o.push_back(B.gate(AND, Q[k], nz));
      break;
    }
    case kUnitCmp:
    case kUnitSubs:
    case kUnitAdds: {
      const bool add = unit == kUnitAdds;
      std::vector<Ref> bb(w);
      for (int i = 0; i < w; ++i) bb[i] = add ? b[i] : !b[i];
      AdderOut r = add ? kogge_stone(B, a, bb, 0, Ref{}) : kogge_stone(B, a, bb, 1, Ref{});
      const Ref s = r.sum[w - 1];
      const Ref N = s;
      const Ref Z = !or_tree(B, r.sum);
      const Ref C = r.carry;
      // §6: V = (!x !y s) + (x y !s) for the added operands x = a, y = b
      // (ADDS) or y = NOT b (CMP, SUBS), in gates on a and b.
      const Ref x1 = B.gate(add ? NOR : ANDNY, a[w - 1], b[w - 1]);
      const Ref x2 = B.gate(AND, x1, s);
      const Ref y1 = B.gate(add ? AND : ANDYN, a[w - 1], b[w - 1]);
      const Ref y2 = B.gate(ANDYN, y1, s);
      const Ref V = B.gate(OR, x2, y2);
      if (unit != kUnitCmp) o = r.sum;
      o.push_back(N);
      o.push_back(Z);
      o.push_back(C);
      o.push_back(V);
      break;
    }
    case kUnitSmull:
    case kUnitUmull:
      o = full_multiplier(B, a, b, unit == kUnitSmull);
      break;
    case kUnitCsel: {
      const Ref N = B.in(2 * w), Z = B.in(2 * w + 1), C = B.in(2 * w + 2), V = B.in(2 * w + 3);
      const Ref c = condition(B, cond, N, Z, C, V);
      for (int j = 0; j < w; ++j) o.push_back(B.mux(c, a[j], b[j]));
      break;
    }
    default:
      return false;
  }
  *out = B.finish(o);
  return true;
}

}  // namespace ce
