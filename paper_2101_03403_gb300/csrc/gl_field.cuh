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

// a + b mod p.  An overflow past 2^64 is worth 2^64 = eps (mod p); adding eps
// back can overflow once more only when the wrapped sum is >= p.
__device__ __forceinline__ uint64_t add(uint64_t a, uint64_t b) {
  uint64_t s = a + b;
  if (s < a) {
    s += kEps;
    if (s < kEps) s += kEps;
  }
  return s;
}

// a - b mod p.  A borrow is worth -2^64 = -eps (mod p).
__device__ __forceinline__ uint64_t sub(uint64_t a, uint64_t b) {
  uint64_t d = a - b;
  if (a < b) {
    const uint64_t d2 = d - kEps;
    d = (d < kEps) ? d2 - kEps : d2;
  }
  return d;
}

// hi * 2^64 + lo mod p, using 2^64 = 2^32 - 1 and 2^96 = -1:
// value = lo - hi_hi + hi_lo * (2^32 - 1).  Each step needs at most one
// correction (the bounds: lo - hi_hi + 2^64 > eps; hi_lo * eps < 2^64 - eps).
__device__ __forceinline__ uint64_t reduce128(uint64_t hi, uint64_t lo) {
  const uint64_t hh = hi >> 32;
  const uint64_t hl = hi & kEps;
  uint64_t t0 = lo - hh;
  if (lo < hh) t0 -= kEps;
  const uint64_t t1 = (hl << 32) - hl;
  uint64_t r = t0 + t1;
  if (r < t1) r += kEps;
  return r;
}

__device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t b) {
  return reduce128(__umul64hi(a, b), a * b);
}

__device__ __forceinline__ uint64_t neg(uint64_t a) { return sub(0ull, a); }

// x * 2^s mod p for a shift known after unrolling (s in [0, 192)).
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
  } else if (s < 64) {
    r = reduce128(x >> (64 - s), x << s);
  } else {
    // x * 2^s = y * 2^64 with y = x * 2^(s-64); y * 2^64 = y * (2^32 - 1).
    const int t = s - 64;
    const uint64_t y = (t == 0) ? x : reduce128(x >> (64 - t), x << t);
    const uint64_t lo = y << 32, hi = y >> 32;
    r = reduce128(hi - (lo < y ? 1ull : 0ull), lo - y);
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
