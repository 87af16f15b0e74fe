// Exact negacyclic products over Z_{2^32}[X]/(X^1024 + 1): a 1024-point
// number-theoretic transform in the two-prime residue system of
// rns_arith.h, computed by 128 threads for a pair of polynomials (the blind
// rotation's external product, §3 "TFHE Library": one CMux per key bit).
//
// Transform structure (psi a primitive 2048-th root of unity mod p): the
// negacyclic transform X_k = sum_n x_n psi^(n (2k+1)) split as
// n = n1 + 64 n2, k = k2 + 16 k1:
//   A  : pre-twist psi^(64 n2), 16-point transform over n2 (root psi^128),
//        twist psi^(n1 (2 k2 + 1));
//   C1 : 8-point transforms over b (n1 = a + 8 b, root psi^256), twiddle
//        psi^(32 a c);
//   C2 : 8-point transforms over a, k1 = c + 8 d.
// Thread t of a 128-thread group ends owning positions
// k = (t & 15) + 16 ((t >> 4) + 8 d), d = 0..7, of both polynomials, so the
// pointwise products need no exchange.  Phases exchange data through a
// shared buffer of [2][16][65] (residue pairs; the padding keeps every warp
// access conflict-free).  The inverse runs the phases backwards with
// inverse roots; the 1/1024 scale is folded into its twist table.
#pragma once

#include "rns_arith.h"

// Transform code reads the uniform table, which lives in constant memory on
// the device; it is compiled for the device only (or for a host build of this
// header without CUDA).
#ifdef __CUDACC__
#define RNS_TD __device__ __forceinline__
#else
#define RNS_TD inline
#endif

// The uniform factor table, visible to the transform code below as RNS_U.
#if defined(__CUDACC__)
__constant__ rns::Uniform c_rns_uniform = rns::make_uniform();
#define RNS_U c_rns_uniform
#else
constexpr rns::Uniform k_rns_uniform = rns::make_uniform();
#define RNS_U k_rns_uniform
#endif

namespace rns {

constexpr int kRow = 65;                 // padded row of the transpose buffer
constexpr int kBufWords = 2 * 16 * kRow; // residue pairs per 128-thread group

RNS_HD constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1) << (bits - 1 - i);
  return r;
}
RNS_HD constexpr int ilog2(int m) { return m <= 1 ? 0 : 1 + ilog2(m >> 1); }

template <int M, int DIR, int Q>
RNS_TD Tw root(int e) {
  if (M == 16) return RNS_U.r16[DIR][Q][e];
  return RNS_U.r8[DIR][Q][e];
}

#ifdef RNS_RANGE_CHECK  // host builds of this header may check every lazy bound
#define RNS_EXPECT(x, bound) rns_range_check((x) < (bound))
#else
#define RNS_EXPECT(x, bound) ((void)0)
#endif

// In-register transform V[k] = sum_n v[n] w^(n k), w = psi^(+-2048/M)
// (DIR 0: +, 1: -).  Radix-2 decimation in frequency; the bit-reversed
// output order is undone by renaming registers.  Inputs lie in [0, 4p), or
// in [0, 2p) when IN2P (then the first stage needs no reduction); outputs
// lie in [0, 4p), except outputs k of the last stage whose bit in FOLD is
// clear: those are left in [0, 8p) for a consumer that multiplies them
// (a Shoup product or a Montgomery sum accepts any 32-bit value).
template <int M, int DIR, int Q, bool IN2P = false, unsigned FOLD = 0xFFFFu>
RNS_TD void dft(uint32_t (&v)[M]) {
  constexpr int LOG = ilog2(M);
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
    const int len = M >> (st + 1);
    const bool first = IN2P && st == 0, last = st == LOG - 1;
    const uint32_t off = (first ? 2u : 4u) * P<Q>();
#pragma unroll
    for (int j0 = 0; j0 < M; j0 += 2 * len) {
#pragma unroll
      for (int i = 0; i < len; ++i) {
        const int e = i * (M / (2 * len));
        uint32_t &a = v[j0 + i], &b = v[j0 + i + len];
        RNS_EXPECT(a, (first ? 2u : 4u) * P<Q>());
        RNS_EXPECT(b, (first ? 2u : 4u) * P<Q>());
        const uint32_t s = a + b, d = a + off - b;
        const bool fold_s = !first && (!last || ((FOLD >> bitrev(j0 + i, LOG)) & 1u));
        const bool fold_d = !first && (!last || ((FOLD >> bitrev(j0 + i + len, LOG)) & 1u));
        a = fold_s ? fold<Q, 4>(s) : s;
        if (e == 0)
          b = fold_d ? fold<Q, 4>(d) : d;
        else
          b = shoup<Q>(d, root<M, DIR, Q>(e));
      }
    }
  }
  uint32_t t[M];
#pragma unroll
  for (int k = 0; k < M; ++k) t[k] = v[bitrev(k, LOG)];
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] = t[k];
}

RNS_TD uint4 load_tw(const uint4 *p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// Pre-twist of a phase-A input u (in [0, 4p)) at row n2.
template <int Q>
RNS_TD uint32_t pretwist(uint32_t u, int n2) {
  return n2 == 0 ? u : shoup<Q>(u, RNS_U.pre[0][Q][n2]);
}

// ------------------------------------------------------------ forward ---
// tw_fwd: uint4 {w0, w0', w1, w1'} of psi^(n1 (2 k2 + 1)) at [k2 * 64 + n1].

// Phase A: thread (Pp, n1) = (t >> 6, t & 63) holds v[q][n2] = x_Pp[n1 + 64 n2]
// mod p_q, pre-twisted.
RNS_TD void fwd_phase_a(uint32_t (&v)[2][16], uint2 *buf, int t, const uint4 *tw_fwd) {
  const int Pp = t >> 6, n1 = t & 63;
  dft<16, 0, 0, true, 0u>(v[0]);  // every output is twisted
  dft<16, 0, 1, true, 0u>(v[1]);
  uint2 *col = buf + Pp * 16 * kRow + n1;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const uint4 T = load_tw(tw_fwd + k2 * 64 + n1);
    col[k2 * kRow] = make_uint2(shoup<0>(v[0][k2], T.x, T.y), shoup<1>(v[1][k2], T.z, T.w));
  }
}

// Phase C1 for warp wg: lane -> (Pp, k2) = (lane >> 4, lane & 15), a in
// {2 wg, 2 wg + 1} (warp-uniform).  Reads positions a + 8 b of its row and
// writes positions 8 c + a: touched by no other thread, so in place.
RNS_TD void fwd_phase_c1(uint2 *buf, int wg, int lane) {
  uint2 *row = buf + ((lane >> 4) * 16 + (lane & 15)) * kRow;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int a = 2 * wg + j;
    uint32_t u0[8], u1[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint2 x = row[a + 8 * b];
      u0[b] = x.x;
      u1[b] = x.y;
    }
    dft<8, 0, 0, true, 1u>(u0);  // outputs c >= 1 are multiplied below
    dft<8, 0, 1, true, 1u>(u1);
    row[a] = make_uint2(u0[0], u1[0]);
#pragma unroll
    for (int c = 1; c < 8; ++c)
      row[c * 8 + a] = make_uint2(shoup<0>(u0[c], RNS_U.c1[0][0][a * 8 + c]),
                                  shoup<1>(u1[c], RNS_U.c1[0][1][a * 8 + c]));
  }
}

// Phase C2: thread (k2, c) = (t & 15, t >> 4), both polynomials.  Outputs
// lie in [0, 8p) (products accept them).
RNS_TD void fwd_phase_c2(uint32_t (&X)[2][2][8], const uint2 *buf, int t) {
  const int k2 = t & 15, c = t >> 4;
#pragma unroll
  for (int Pp = 0; Pp < 2; ++Pp) {
    const uint2 *row = buf + (Pp * 16 + k2) * kRow + c * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const uint2 x = row[a];
      X[0][Pp][a] = x.x;
      X[1][Pp][a] = x.y;
    }
    dft<8, 0, 0, false, 0u>(X[0][Pp]);  // outputs feed products: [0, 8p)
    dft<8, 0, 1, false, 0u>(X[1][Pp]);
  }
}

// ------------------------------------------------------------ inverse ---
// tw_inv: psi^(-n1 (2 k2 + 1)) / 1024 at [k2 * 64 + n1].

RNS_TD void inv_phase_c2(uint32_t (&X)[2][2][8], uint2 *buf, int t) {
  const int k2 = t & 15, c = t >> 4;
#pragma unroll
  for (int Pp = 0; Pp < 2; ++Pp) {
    dft<8, 1, 0>(X[0][Pp]);
    dft<8, 1, 1>(X[1][Pp]);
    uint2 *row = buf + (Pp * 16 + k2) * kRow + c * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) row[a] = make_uint2(X[0][Pp][a], X[1][Pp][a]);
  }
}

RNS_TD void inv_phase_c1(uint2 *buf, int wg, int lane) {
  uint2 *row = buf + ((lane >> 4) * 16 + (lane & 15)) * kRow;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int a = 2 * wg + j;
    uint32_t u0[8], u1[8];
    {
      const uint2 x = row[a];
      u0[0] = x.x;
      u1[0] = x.y;
    }
#pragma unroll
    for (int c = 1; c < 8; ++c) {
      const uint2 x = row[c * 8 + a];
      u0[c] = shoup<0>(x.x, RNS_U.c1[1][0][a * 8 + c]);
      u1[c] = shoup<1>(x.y, RNS_U.c1[1][1][a * 8 + c]);
    }
    dft<8, 1, 0, false, 0u>(u0);  // phase A multiplies every output
    dft<8, 1, 1, false, 0u>(u1);
#pragma unroll
    for (int b = 0; b < 8; ++b) row[a + 8 * b] = make_uint2(u0[b], u1[b]);
  }
}

// Inverse phase A: v[q][n2] receives x_Pp[n1 + 64 n2] mod p_q in [0, 4p).
RNS_TD void inv_phase_a(uint32_t (&v)[2][16], const uint2 *buf, int t, const uint4 *tw_inv) {
  const int Pp = t >> 6, n1 = t & 63;
  const uint2 *col = buf + Pp * 16 * kRow + n1;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const uint4 T = load_tw(tw_inv + k2 * 64 + n1);
    const uint2 x = col[k2 * kRow];
    v[0][k2] = shoup<0>(x.x, T.x, T.y);
    v[1][k2] = shoup<1>(x.y, T.z, T.w);
  }
  dft<16, 1, 0, true, 1u>(v[0]);  // outputs n2 >= 1 are multiplied below
  dft<16, 1, 1, true, 1u>(v[1]);
#pragma unroll
  for (int n2 = 1; n2 < 16; ++n2) {
    v[0][n2] = shoup<0>(v[0][n2], RNS_U.pre[1][0][n2]);
    v[1][n2] = shoup<1>(v[1][n2], RNS_U.pre[1][1][n2]);
  }
}

// ------------------------------------------------- group-level wrappers ---
#ifdef __CUDACC__
// Barrier `id` over `count` threads (all groups of a block share one barrier
// so that every warp of the block runs the same code region at a time).
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Forward transform of two polynomials; v holds this thread's pre-twisted
// phase-A inputs in [0, 2p) (clobbered); X receives the eight positions of
// each, in [0, 8p).
__device__ __forceinline__ void forward(uint32_t (&v)[2][16], uint32_t (&X)[2][2][8], uint2 *buf,
                                        int t, int bar, int nthr, const uint4 *tw_fwd) {
  named_bar(bar, nthr);  // the buffer is free
  fwd_phase_a(v, buf, t, tw_fwd);
  named_bar(bar, nthr);
  fwd_phase_c1(buf, t >> 5, t & 31);
  named_bar(bar, nthr);
  fwd_phase_c2(X, buf, t);
}

// Inverse transform: X (clobbered, values in [0, 4p)) holds this thread's
// positions of both polynomials; v receives x_Pp[n1 + 64 n2].
__device__ __forceinline__ void inverse(uint32_t (&X)[2][2][8], uint32_t (&v)[2][16], uint2 *buf,
                                        int t, int bar, int nthr, const uint4 *tw_inv) {
  named_bar(bar, nthr);
  inv_phase_c2(X, buf, t);
  named_bar(bar, nthr);
  inv_phase_c1(buf, t >> 5, t & 31);
  named_bar(bar, nthr);
  inv_phase_a(v, buf, t, tw_inv);
}
#endif

}  // namespace rns
