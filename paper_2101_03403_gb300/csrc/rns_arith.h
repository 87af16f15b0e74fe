// Two-prime residue arithmetic for the exact negacyclic products of the
// blind rotation's external product (§3 "TFHE Library": one CMux per key
// bit); the transform built on it is in rns_ntt.cuh.
//
// A digit polynomial (|d| <= 512) times a key polynomial (lifted to
// [-2^31, 2^31)) summed over the six TRGSW rows of a CMux step is an integer
// of magnitude below 6 * 1024 * 2^9 * 2^31 < 2^53.6; the two primes' product
// P ~ 2^56 exceeds twice that, so the centred residue mod P (Garner's
// reconstruction from the two residues) is the exact integer and its low 32
// bits the torus result.
//
// Arithmetic per prime p (all 32-bit):
//   - values are kept lazily below B p for a bound B <= 16 tracked at compile
//     time (p < 2^28, so 16 p fits in 32 bits; rns_ntt.cuh);
//   - multiplication by a fixed factor w uses Shoup's precomputed quotient
//     w' = floor(w 2^32 / p): x w - umulhi(x, w') p lies in [0, 2p) for any
//     32-bit x (three integer multiply-adds);
//   - key products are accumulated as 64-bit sums of 32 x 32-bit products
//     and reduced once by Montgomery's method (key stored times 2^32 mod p).
//
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#define RNS_HD __host__ __device__ __forceinline__
#define RNS_CX __host__ __device__ constexpr
#else
#define RNS_HD inline
#define RNS_CX constexpr
struct uint2 {
  uint32_t x, y;
};
struct uint4 {
  uint32_t x, y, z, w;
};
inline uint2 make_uint2(uint32_t x, uint32_t y) { return uint2{x, y}; }
#endif

namespace rns {

// ------------------------------------------------------------ constants ---

template <int Q>
RNS_HD constexpr uint32_t P() {
  return Q == 0 ? 0x0FFF0001u : 0x0FFEF801u;  // 2^28 - 2^16 + 1, 2^28 - 2^16 - 2^11 + 1
}
template <int Q>
RNS_HD constexpr uint32_t Psi() {  // primitive 2048-th roots of unity
  return Q == 0 ? 135902522u : 16675871u;
}

RNS_CX uint32_t mulm(uint32_t a, uint32_t b, uint32_t p) {
  return uint32_t(uint64_t(a) * b % p);
}
RNS_CX uint32_t powm(uint32_t a, uint64_t e, uint32_t p) {
  uint32_t r = 1;
  while (e) {
    if (e & 1) r = mulm(r, a, p);
    a = mulm(a, a, p);
    e >>= 1;
  }
  return r;
}
RNS_CX uint32_t invm(uint32_t a, uint32_t p) { return powm(a, p - 2, p); }
RNS_CX uint32_t shoup_of(uint32_t w, uint32_t p) { return uint32_t((uint64_t(w) << 32) / p); }
// -p^-1 mod 2^32 (Newton's iteration doubles the correct low bits).
RNS_CX uint32_t neg_inv32(uint32_t p) {
  uint32_t x = p;
  for (int i = 0; i < 5; ++i) x *= 2u - p * x;
  return 0u - x;
}
template <int Q>
RNS_HD constexpr uint32_t NInv() {
  return Q == 0 ? neg_inv32(P<0>()) : neg_inv32(P<1>());
}

static_assert(powm(Psi<0>(), 1024, P<0>()) == P<0>() - 1, "psi_0 has order 2048");
static_assert(powm(Psi<1>(), 1024, P<1>()) == P<1>() - 1, "psi_1 has order 2048");
static_assert(uint32_t(P<0>() * neg_inv32(P<0>())) == 0xFFFFFFFFu, "Montgomery constant 0");
static_assert(uint32_t(P<1>() * neg_inv32(P<1>())) == 0xFFFFFFFFu, "Montgomery constant 1");

// Garner: S = r0 + p0 ((r1 - r0) p0^-1 mod p1) in [0, P).
constexpr uint64_t kPP = uint64_t(0x0FFF0001u) * 0x0FFEF801u;
constexpr uint32_t kCrt = invm(0x0FFF0001u % 0x0FFEF801u, 0x0FFEF801u);
constexpr uint32_t kCrtP = shoup_of(kCrt, 0x0FFEF801u);
static_assert(kPP > (uint64_t(6 * 1024) << 41), "P exceeds twice the largest |exact sum|");

// Per-thread factor table (global memory, L1-resident), entries uint4
// {w mod p0, its Shoup quotient, w mod p1, its Shoup quotient}:
//   [0, 1024)      forward twist psi^(n1 (2 k2 + 1)) at k2 * 64 + n1,
//   [1024, 2048)   inverse twist psi^(-n1 (2 k2 + 1)) / 1024,
//   [2048, 2112)   forward middle-phase twiddle psi^(32 a c) at a * 8 + c,
//   [2112, 2176)   inverse middle-phase twiddle psi^(-32 a c).
constexpr int kTwInv = 1024, kTwC1Fwd = 2048, kTwC1Inv = 2112, kTwEntries = 2176;

struct Tw {
  uint32_t w, wp;
};

// Warp-uniform factors, indexed by compile-time constants after unrolling
// (constant-bank operands on the device).  dir 0 = forward, 1 = inverse.
struct Uniform {
  Tw pre[2][2][16];  // [dir][q][n2]: psi^(+-64 n2)
  Tw r16[2][2][8];   // [dir][q][e]: psi^(+-128 e)
  Tw r8[2][2][4];    // [dir][q][e]: psi^(+-256 e)
};

constexpr Uniform make_uniform() {
  Uniform u{};
  const uint32_t ps[2] = {P<0>(), P<1>()};
  const uint32_t rt[2] = {Psi<0>(), Psi<1>()};
  for (int q = 0; q < 2; ++q) {
    const uint32_t p = ps[q];
    const uint32_t root[2] = {rt[q], invm(rt[q], p)};
    for (int dir = 0; dir < 2; ++dir) {
      const uint32_t r = root[dir];
      for (int n2 = 0; n2 < 16; ++n2) {
        const uint32_t w = powm(r, 64u * n2, p);
        u.pre[dir][q][n2] = Tw{w, shoup_of(w, p)};
      }
      for (int e = 0; e < 8; ++e) {
        const uint32_t w = powm(r, 128u * e, p);
        u.r16[dir][q][e] = Tw{w, shoup_of(w, p)};
      }
      for (int e = 0; e < 4; ++e) {
        const uint32_t w = powm(r, 256u * e, p);
        u.r8[dir][q][e] = Tw{w, shoup_of(w, p)};
      }
    }
  }
  return u;
}

// ----------------------------------------------------------- arithmetic ---

RNS_HD uint32_t mulhi(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return uint32_t((uint64_t(a) * b) >> 32);
#endif
}

RNS_HD uint32_t umin(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return min(a, b);
#else
  return a < b ? a : b;
#endif
}

// x w mod p in [0, 2p) for any 32-bit x.
template <int Q>
RNS_HD uint32_t shoup(uint32_t x, uint32_t w, uint32_t wp) {
  return x * w - mulhi(x, wp) * P<Q>();
}
template <int Q>
RNS_HD uint32_t shoup(uint32_t x, Tw t) {
  return shoup<Q>(x, t.w, t.wp);
}

// [0, 2 m p) -> [0, m p) by one conditional subtraction (unsigned minimum:
// below m p the difference wraps above the value).
template <int Q, int M>
RNS_HD uint32_t fold(uint32_t s) {
  return umin(s, s - uint32_t(M) * P<Q>());
}

// x 2^-32 mod p (Montgomery) for x < 2^64 - 2^32 p: the result lies below
// x / 2^32 + p (below 2p for x < 2^32 p).
template <int Q>
RNS_HD uint32_t redc(uint64_t x) {
  const uint32_t m = uint32_t(x) * NInv<Q>();
  return uint32_t((x + uint64_t(m) * P<Q>()) >> 32);
}

// Low 32 bits of the centred integer V (|V| < P/2) with residues r0 (mod p0)
// and r1 (mod p1), each given in [0, 4p).  Garner's formula works on any
// representatives: h = (r1 - r0) p0^-1 mod p1 (the offset 5 p1 > 4 p0 keeps
// the difference positive, below 9 p1 < 2^32), S = r0 + h p0 = V (mod P) with
// S in [0, P + 3 p0); V = S - P exactly when S > P/2 (for S >= P that is the
// representative S - P in [0, 3 p0)).
RNS_HD uint32_t lift32(uint32_t r0, uint32_t r1) {
  uint32_t h = shoup<1>(r1 + 5 * P<1>() - r0, kCrt, kCrtP);
  h = fold<1, 1>(h);
  const uint64_t s = r0 + uint64_t(h) * P<0>();
  return uint32_t(s) - (s > (kPP >> 1) ? uint32_t(kPP) : 0u);
}

// x 2^32 mod p: redc(x R2) for R2 = 2^64 mod p (the Montgomery form in
// which the transform-domain key is stored).
template <int Q>
RNS_HD uint32_t to_mont(uint32_t x) {
  constexpr uint32_t r1 = uint32_t((uint64_t(1) << 32) % P<Q>());
  constexpr uint32_t r2 = mulm(r1, r1, P<Q>());
  return redc<Q>(uint64_t(x) * r2);
}

// Signed 32-bit integer to [0, p).
template <int Q>
RNS_HD uint32_t from_i32(int32_t v) {
  const int64_t r = int64_t(v) % int64_t(P<Q>());
  return uint32_t(r < 0 ? r + P<Q>() : r);
}

}  // namespace rns

