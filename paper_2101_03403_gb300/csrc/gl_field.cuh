// Arithmetic in the prime field F_p, p = 2^64 - 2^32 + 1, on the GPU.
//
// The negacyclic products of the blind rotation (digit polynomials times
// bootstrapping-key polynomials, exact integers below 2^54 in magnitude) are
// computed by a number-theoretic transform over this field: the result mod p,
// read as a signed value, is the exact integer, whose low 32 bits are the
// torus result.  p has 2^32 | p - 1, so 2048-th roots of unity exist; 2 has
// multiplicative order 192 (2^96 = -1), so every root of unity of order
// dividing 64 is a power of two and multiplying by it is a shift plus a
// cheap reduction.  Elements are kept in [0, 2^64) (not necessarily below p).
#pragma once

#include <cstdint>

namespace gl {

constexpr uint64_t kP = 0xFFFFFFFF00000001ull;
constexpr uint64_t kEps = 0xFFFFFFFFull;  // 2^64 mod p

// The operations below are written as explicit carry chains (PTX add.cc /
// addc / sub.cc / subc): every correction is an addition of a carry-derived
// mask, so no 64-bit comparison or select is needed.  Results are in
// [0, 2^64) and congruent mod p; inputs may be any value in [0, 2^64).

// a + b mod p.  An overflow past 2^64 is worth 2^64 = eps (mod p); adding eps
// back can overflow once more only when the wrapped sum is >= p, and then
// the value is below eps, so a third addition of eps cannot overflow.
__device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 a0, a1, b0, b1, s0, s1, c, m, z;\n\t"
      "mov.b64 {a0, a1}, %1;\n\t"
      "mov.b64 {b0, b1}, %2;\n\t"
      "mov.u32 z, 0;\n\t"
      "add.cc.u32 s0, a0, b0;\n\t"
      "addc.cc.u32 s1, a1, b1;\n\t"
      "addc.u32 c, z, z;\n\t"
      "mul.lo.u32 m, c, 0xFFFFFFFF;\n\t"
      "add.cc.u32 s0, s0, m;\n\t"
      "addc.cc.u32 s1, s1, z;\n\t"
      "addc.u32 c, z, z;\n\t"
      "mul.lo.u32 m, c, 0xFFFFFFFF;\n\t"
      "add.cc.u32 s0, s0, m;\n\t"
      "addc.u32 s1, s1, z;\n\t"
      "mov.b64 %0, {s0, s1};\n\t"
      "}"
      : "=l"(r)
      : "l"(a), "l"(b));
  return r;
}

// a - b mod p.  A borrow is worth -2^64 = -eps (mod p); subtracting eps from
// the wrapped difference can borrow once more only when it is below eps,
// and then a second subtraction of eps cannot borrow.
__device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 a0, a1, b0, b1, d0, d1, w, z;\n\t"
      "mov.b64 {a0, a1}, %1;\n\t"
      "mov.b64 {b0, b1}, %2;\n\t"
      "mov.u32 z, 0;\n\t"
      "sub.cc.u32 d0, a0, b0;\n\t"
      "subc.cc.u32 d1, a1, b1;\n\t"
      "subc.u32 w, z, z;\n\t"
      "sub.cc.u32 d0, d0, w;\n\t"
      "subc.cc.u32 d1, d1, z;\n\t"
      "subc.u32 w, z, z;\n\t"
      "sub.cc.u32 d0, d0, w;\n\t"
      "subc.u32 d1, d1, z;\n\t"
      "mov.b64 %0, {d0, d1};\n\t"
      "}"
      : "=l"(r)
      : "l"(a), "l"(b));
  return r;
}

// hi * 2^64 + lo mod p, using 2^64 = 2^32 - 1 and 2^96 = -1:
// value = lo - hi_hi + hi_lo * (2^32 - 1).  The subtraction needs at most one
// correction (lo - hi_hi + 2^64 > eps); hi_lo * eps = hi_lo * 2^32 - hi_lo is
// below 2^64 - eps, so the final addition needs at most one correction.
__device__ __forceinline__ uint64_t reduce128(uint64_t hi, uint64_t lo) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 l0, l1, h0, h1, t0, t1, u0, u1, w, z;\n\t"
      ".reg .u64 u;\n\t"
      "mov.b64 {l0, l1}, %2;\n\t"
      "mov.b64 {h0, h1}, %1;\n\t"
      "mov.u32 z, 0;\n\t"
      "sub.cc.u32 t0, l0, h1;\n\t"
      "subc.cc.u32 t1, l1, z;\n\t"
      "subc.u32 w, z, z;\n\t"
      "sub.cc.u32 t0, t0, w;\n\t"
      "subc.u32 t1, t1, z;\n\t"
      "mul.wide.u32 u, h0, 0xFFFFFFFF;\n\t"
      "mov.b64 {u0, u1}, u;\n\t"
      "add.cc.u32 t0, t0, u0;\n\t"
      "addc.cc.u32 t1, t1, u1;\n\t"
      "addc.u32 w, z, z;\n\t"
      "mul.lo.u32 w, w, 0xFFFFFFFF;\n\t"
      "add.cc.u32 t0, t0, w;\n\t"
      "addc.u32 t1, t1, z;\n\t"
      "mov.b64 %0, {t0, t1};\n\t"
      "}"
      : "=l"(r)
      : "l"(hi), "l"(lo));
  return r;
}

// y0 + 2^32 y1 + 2^64 y2 mod p = (y1:y0) + y2 * eps (y2 < 2^32); the
// product y2 * eps < 2^64 - eps, so one correction suffices.
__device__ __forceinline__ uint64_t reduce96(uint32_t y0, uint32_t y1, uint32_t y2) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 t0, t1, u0, u1, w, z;\n\t"
      ".reg .u64 u;\n\t"
      "mov.u32 z, 0;\n\t"
      "mul.wide.u32 u, %3, 0xFFFFFFFF;\n\t"
      "mov.b64 {u0, u1}, u;\n\t"
      "add.cc.u32 t0, %1, u0;\n\t"
      "addc.cc.u32 t1, %2, u1;\n\t"
      "addc.u32 w, z, z;\n\t"
      "mul.lo.u32 w, w, 0xFFFFFFFF;\n\t"
      "add.cc.u32 t0, t0, w;\n\t"
      "addc.u32 t1, t1, z;\n\t"
      "mov.b64 %0, {t0, t1};\n\t"
      "}"
      : "=l"(r)
      : "r"(y0), "r"(y1), "r"(y2));
  return r;
}

// x * 2^s as 96 bits (y0, y1, y2) for 0 <= s < 32, by two 32x32->64
// multiply-adds (the integer multiply-add pipe, not the shifter).
__device__ __forceinline__ void shl96(uint64_t x, int s, uint32_t &y0, uint32_t &y1, uint32_t &y2) {
  const uint32_t x0 = static_cast<uint32_t>(x), x1 = static_cast<uint32_t>(x >> 32);
  const uint32_t f = 1u << s;
  const uint64_t lo = static_cast<uint64_t>(x0) * f;
  const uint64_t hi = static_cast<uint64_t>(x1) * f + (lo >> 32);
  y0 = static_cast<uint32_t>(lo);
  y1 = static_cast<uint32_t>(hi);
  y2 = static_cast<uint32_t>(hi >> 32);
}

// x + a * b + c * d mod p with one reduction: the two 128-bit products and
// x are summed in 130 bits (carry word k <= 2); with 2^96 = -1 and
// 2^128 = -2^32 the value is lo - (h1 + k * 2^32) + h0 * eps, where the
// subtrahend is below 2^34 (one borrow correction) and h0 * eps below
// 2^64 - eps (one carry correction).
__device__ __forceinline__ uint64_t mac2(uint64_t x, uint64_t a, uint64_t b, uint64_t c,
                                         uint64_t d) {
  const uint64_t lo1 = a * b, hi1 = __umul64hi(a, b);
  const uint64_t lo2 = c * d, hi2 = __umul64hi(c, d);
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 a0, a1, a2, a3, b0, b1, b2, b3, x0, x1, k, w, z, u0, u1;\n\t"
      ".reg .u64 u;\n\t"
      "mov.u32 z, 0;\n\t"
      "mov.b64 {a0, a1}, %1;\n\t"
      "mov.b64 {a2, a3}, %2;\n\t"
      "mov.b64 {b0, b1}, %3;\n\t"
      "mov.b64 {b2, b3}, %4;\n\t"
      "mov.b64 {x0, x1}, %5;\n\t"
      "add.cc.u32 a0, a0, b0;\n\t"
      "addc.cc.u32 a1, a1, b1;\n\t"
      "addc.cc.u32 a2, a2, b2;\n\t"
      "addc.cc.u32 a3, a3, b3;\n\t"
      "addc.u32 k, z, z;\n\t"
      "add.cc.u32 a0, a0, x0;\n\t"
      "addc.cc.u32 a1, a1, x1;\n\t"
      "addc.cc.u32 a2, a2, z;\n\t"
      "addc.cc.u32 a3, a3, z;\n\t"
      "addc.u32 k, k, z;\n\t"
      // t = lo - (a3 + k * 2^32); on borrow add p (= subtract eps)
      "sub.cc.u32 a0, a0, a3;\n\t"
      "subc.cc.u32 a1, a1, k;\n\t"
      "subc.u32 w, z, z;\n\t"
      "sub.cc.u32 a0, a0, w;\n\t"
      "subc.u32 a1, a1, z;\n\t"
      // + a2 * eps
      "mul.wide.u32 u, a2, 0xFFFFFFFF;\n\t"
      "mov.b64 {u0, u1}, u;\n\t"
      "add.cc.u32 a0, a0, u0;\n\t"
      "addc.cc.u32 a1, a1, u1;\n\t"
      "addc.u32 w, z, z;\n\t"
      "mul.lo.u32 w, w, 0xFFFFFFFF;\n\t"
      "add.cc.u32 a0, a0, w;\n\t"
      "addc.u32 a1, a1, z;\n\t"
      "mov.b64 %0, {a0, a1};\n\t"
      "}"
      : "=l"(r)
      : "l"(lo1), "l"(hi1), "l"(lo2), "l"(hi2), "l"(x));
  return r;
}

// a * b + c * d mod p with one reduction.
__device__ __forceinline__ uint64_t mul2_add(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
  return mac2(0, a, b, c, d);
}

__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
  return reduce128(__umul64hi(a, b), a * b);
}

__device__ __forceinline__ uint64_t neg(uint64_t a) { return sub(0ull, a); }

// x * 2^s mod p for a shift known after unrolling (s in [0, 192)).
// 2^96 = -1 folds s into [0, 96); x * 2^s is formed by multiply-adds:
// s < 32: 96-bit product, reduced with 2^64 = eps; 32 <= s < 64: the
// 96-bit product x * 2^(s-32) moved up one 32-bit limb (a 128-bit value);
// 64 <= s < 96: y = x * 2^(s-64) reduced, then y * 2^64 = y * eps.
__device__ __forceinline__ uint64_t mul_pow2(uint64_t x, int s) {
  s %= 192;
  if (s < 0) s += 192;
  bool negate = false;
  if (s >= 96) {  // 2^96 = -1
    s -= 96;
    negate = true;
  }
  uint64_t r;
  if (s == 0) {
    r = x;
  } else if (s < 32) {
    uint32_t y0, y1, y2;
    shl96(x, s, y0, y1, y2);
    r = reduce96(y0, y1, y2);
  } else if (s < 64) {
    uint32_t y0, y1, y2;
    shl96(x, s - 32, y0, y1, y2);
    // value y0 * 2^32 + y1 * 2^64 + y2 * 2^96
    r = reduce128((static_cast<uint64_t>(y2) << 32) | y1, static_cast<uint64_t>(y0) << 32);
  } else {
    const int t = s - 64;
    uint64_t y = x;
    if (t) {
      uint32_t y0, y1, y2;
      shl96(x, t, y0, y1, y2);
      y = reduce96(y0, y1, y2);
    }
    // y * 2^64 = y * eps = y * 2^32 - y
    const uint32_t q0 = static_cast<uint32_t>(y), q1 = static_cast<uint32_t>(y >> 32);
    r = reduce128(q1, (static_cast<uint64_t>(q0) << 32));  // y * 2^32 as 96 bits
    r = sub(r, y);
  }
  return negate ? neg(r) : r;
}

// x * 2^s mod p for a runtime shift s in [0, 192) that is the same across
// the warp: the case branches are uniform, and the shifts are register
// funnel shifts.  Kept out of line of the unrolled code by the compiler's
// choice; one copy serves every call site with a warp-uniform shift.
__device__ __forceinline__ uint64_t mul_pow2_uniform(uint64_t x, int s) {
  bool negate = false;
  if (s >= 96) {
    s -= 96;
    negate = true;
  }
  uint64_t r;
  if (s == 0) {
    r = x;
  } else if (s < 64) {
    r = reduce128(x >> (64 - s), x << s);
  } else {
    const int t = s - 64;
    const uint64_t y = (t == 0) ? x : reduce128(x >> (64 - t), x << t);
    const uint64_t lo = y << 32, hi = y >> 32;
    r = reduce128(hi - (lo < y ? 1ull : 0ull), lo - y);
  }
  return negate ? neg(r) : r;
}

// Signed small integer as a field element.
__device__ __forceinline__ uint64_t from_i32(int32_t v) {
  return v >= 0 ? static_cast<uint64_t>(v) : kP - static_cast<uint64_t>(-static_cast<int64_t>(v));
}

// Low 32 bits of the integer represented by r, when that integer lies in
// (-p/2, p/2): r in [2^63, 2^64) stands for r - p, and p = 1 (mod 2^32).
__device__ __forceinline__ uint32_t lift32(uint64_t r) {
  return static_cast<uint32_t>(r) - static_cast<uint32_t>(r >> 63);
}

}  // namespace gl
