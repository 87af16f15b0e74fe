// Functional units as netlists of bootstrapped gates (host side).
//
// A netlist is built once per (unit, width, condition) and evaluated level by
// level: every gate's level is one more than the highest level of its
// inputs (inputs and constants are level 0), and all gates of one level of
// all in-flight instructions form one batched launch.  NOT, COPY, CONSTANT
// and shifts by a constant are free: they become negation flags or wire
// references (§3: those operations need no bootstrapping).
#pragma once

#include <cstdint>
#include <vector>

namespace ce {

constexpr uint8_t kOpMux = 10;        // besides the ce_gate_op values 0..9
constexpr int32_t kWireFalse = -1;    // the trivial ciphertext (0, -1/8)

// A reference to a wire, possibly negated.  The constant true is the
// negated constant false.
struct Ref {
  int32_t wire = kWireFalse;
  bool neg = false;
};
inline Ref constant(bool v) { return Ref{kWireFalse, v}; }
inline Ref operator!(Ref r) { return Ref{r.wire, !r.neg}; }

// op(a, b) for gates; MUX: s = a, a ? b : c.
struct NGate {
  uint8_t op;
  Ref a, b, c;
  int32_t out;    // wire index written
  int32_t level;  // 1-based
};

struct Netlist {
  int32_t n_inputs = 0;
  int32_t n_wires = 0;               // inputs + gate outputs
  int32_t depth = 0;
  std::vector<NGate> gates;          // ordered by (level, creation order)
  std::vector<int32_t> level_begin;  // gates of level L are [level_begin[L-1], level_begin[L])
  std::vector<Ref> outputs;
  int32_t bootstraps() const;        // binary gate = 1, MUX = 2
};

// Unit identifiers (the C ABI's ce_unit values).
enum Unit : int {
  kUnitAdd = 0,        // Kogge-Stone parallel-prefix adder (§5 "Adder")
  kUnitAddRipple = 1,  // ripple-carry adder
  kUnitSub = 2,        // a + NOT b + 1 (§5 "Subtractor")
  kUnitAnd = 3,        // bitwise AND (§5 "Bitwise operations")
  kUnitOrr = 4,        // bitwise OR
  kUnitLsl = 5,        // barrel shifter, register amount (§5 "Shifter")
  kUnitMul = 6,        // array multiplier, low half (§5 "Multiplier")
  kUnitUdiv = 7,       // non-restoring divider (§5 "Divider"), x / 0 = 0
  kUnitCmp = 8,        // NZCV of a - b (§6 "Conditional Flags")
  kUnitCsel = 9,       // cond(NZCV) ? rn : rm, cond in 0..13 (EQ..LE)
  kUnitLsr = 10,       // logical right shift, register amount (§5 "Logic right shift")
  kUnitAsr = 11,       // arithmetic right shift (§5 "Arithmetic right shift")
  kUnitEor = 12,       // bitwise XOR (§5 "Bitwise operations")
  kUnitOrn = 13,       // bitwise a OR NOT b
  kUnitAdds = 14,      // a + b and its NZCV (flag-setting add, §6)
  kUnitSubs = 15,      // a - b and its NZCV (CMP that keeps the difference)
  kUnitSmull = 16,     // signed a * b, full 2w-bit product (§5 "Signed multiplication")
  kUnitUmull = 17,     // unsigned a * b, full 2w-bit product (§5 "Unsigned multiplication")
  kUnitAddMux = 18,    // ADD with each span combine's carry as one MUX (fewer levels)
  kUnitSubMux = 19,    // SUB likewise
  kUnitMulTree = 20,   // MUL's low half by column compression (a Wallace tree): fewer levels
  kUnitUdivMux = 21,   // UDIV with the MUX-carry adder in every step
  kUnitCount = 22
};

// Inputs: a[width] then b[width] (CSEL: rn[width], rm[width], N, Z, C, V).
// Outputs: width bits (CMP: N, Z, C, V; ADDS/SUBS: width bits then N, Z, C,
// V; SMULL/UMULL: 2 width bits, low half first).  Returns false for a bad
// request.
bool build_unit(int unit, int width, int cond, Netlist *out);

}  // namespace ce
