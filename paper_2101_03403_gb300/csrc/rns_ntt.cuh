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

#include <utility>

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

// Lazy reduction with bounds known at compile time.  Every value is a
// representative below B p for a bound B (a small integer) that is tracked
// per register through a transform: a sum of x < Bx p and y < By p is below
// (Bx + By) p, the difference x + By p - y too, and a Shoup product is below
// 2p whatever its input.  With p < 2^28 any value below 16 p fits in 32 bits,
// so a register is reduced (x -> min(x, x - m p) for x < 2 m p, halving its
// bound) only where a sum would otherwise pass 16 p or a consumer needs a
// smaller bound.  The plan of one M-point transform is computed by constexpr
// code and expanded with template indices, so every reduction and offset is
// a compile-time constant of the unrolled code.
constexpr int kLazyLimit = 16;
static_assert(uint64_t(kLazyLimit) * P<0>() < (uint64_t(1) << 32) &&
                  uint64_t(kLazyLimit) * P<1>() < (uint64_t(1) << 32),
              "16 p must fit in 32 bits");

struct LazyStep {
  int fa, fb;   // reduction multiple m applied to a / b before the butterfly (0: none)
  int ba, bb;   // bounds of a / b entering the butterfly (after those reductions)
  int off;      // the difference is a + off p - b (off = bound of b)
};
template <int M>
struct LazyPlan {
  LazyStep step[4][8];  // [stage][butterfly] (M <= 16)
  int ofold[16][3];     // reductions of output k after the last stage
  int obound[16];       // bound of output k
  bool ok;              // every sum below kLazyLimit p and every output within its limit
};

RNS_CX int lazy_halve(int b) { return (b + 1) / 2; }

// Radix-2 decimation in frequency, butterfly bi of stage st acts on
// registers (a, b) = (g 2 len + i, g 2 len + i + len) with len = M >> (st+1),
// g = bi / len, i = bi % len; twiddle exponent i M / (2 len) (0: none).
template <int M>
RNS_CX LazyPlan<M> make_lazy_plan(int ib0, int ib, int ob0, int ob) {
  LazyPlan<M> P{};
  P.ok = true;
  int B[16] = {};
  for (int k = 0; k < M; ++k) B[k] = k == 0 ? ib0 : ib;
  const int LOG = ilog2(M);
  for (int st = 0; st < LOG; ++st) {
    const int len = M >> (st + 1);
    for (int bi = 0; bi < M / 2; ++bi) {
      const int g = bi / len, i = bi % len;
      const int a = g * 2 * len + i, b = a + len;
      const int e = i * (M / (2 * len));
      LazyStep &S = P.step[st][bi];
      if (B[a] + B[b] > kLazyLimit && B[a] >= B[b]) {
        S.fa = lazy_halve(B[a]);
        B[a] = S.fa;
      }
      if (B[a] + B[b] > kLazyLimit) {
        S.fb = lazy_halve(B[b]);
        B[b] = S.fb;
      }
      if (B[a] + B[b] > kLazyLimit && S.fa == 0) {
        S.fa = lazy_halve(B[a]);
        B[a] = S.fa;
      }
      if (B[a] + B[b] > kLazyLimit) P.ok = false;
      S.ba = B[a];
      S.bb = B[b];
      S.off = B[b];
      const int sum = B[a] + B[b];
      B[a] = sum;
      B[b] = e ? 2 : sum;
    }
  }
  for (int k = 0; k < M; ++k) {
    int x = B[bitrev(k, LOG)];
    const int lim = k == 0 ? ob0 : ob;
    for (int f = 0; f < 3 && x > lim; ++f) {
      P.ofold[k][f] = lazy_halve(x);
      x = P.ofold[k][f];
    }
    if (x > lim) P.ok = false;
    P.obound[k] = x;
  }
  return P;
}

// Bounds of a transform: input 0 below IB0 p, the others below IB p; output
// 0 (after the bit-reversal renaming) is brought below OB0 p, the others
// below OB p.
template <int M, int IB0, int IB, int OB0, int OB>
struct LazyBounds {
  static constexpr LazyPlan<M> plan = make_lazy_plan<M>(IB0, IB, OB0, OB);
  static_assert(plan.ok, "lazy-reduction plan out of range");
};

template <int Q, int Mult>
RNS_HD uint32_t lazy_reduce(uint32_t x) {
  if (Mult == 0) return x;
  return umin(x, x - uint32_t(Mult) * P<Q>());
}

template <int M, int DIR, int Q, class LB, int ST, int BI>
RNS_TD void lazy_bfly(uint32_t (&v)[M]) {
  constexpr int len = M >> (ST + 1);
  constexpr int ia = (BI / len) * 2 * len + BI % len, ib = ia + len;
  constexpr int e = (BI % len) * (M / (2 * len));
  constexpr int fa = LB::plan.step[ST][BI].fa, fb = LB::plan.step[ST][BI].fb;
  constexpr int ba = LB::plan.step[ST][BI].ba, bb = LB::plan.step[ST][BI].bb;
  constexpr int off = LB::plan.step[ST][BI].off;
  uint32_t a = lazy_reduce<Q, fa>(v[ia]), b = lazy_reduce<Q, fb>(v[ib]);
  RNS_EXPECT(a, uint32_t(ba) * P<Q>());
  RNS_EXPECT(b, uint32_t(bb) * P<Q>());
  v[ia] = a + b;
  const uint32_t d = a + uint32_t(off) * P<Q>() - b;
  if constexpr (e == 0)
    v[ib] = d;
  else
    v[ib] = shoup<Q>(d, root<M, DIR, Q>(e));
}

template <int M, int DIR, int Q, class LB, int ST, int... BI>
RNS_TD void lazy_stage(uint32_t (&v)[M], std::integer_sequence<int, BI...>) {
  (lazy_bfly<M, DIR, Q, LB, ST, BI>(v), ...);
}

template <int M, int DIR, int Q, class LB, int... ST>
RNS_TD void lazy_stages(uint32_t (&v)[M], std::integer_sequence<int, ST...>) {
  (lazy_stage<M, DIR, Q, LB, ST>(v, std::make_integer_sequence<int, M / 2>{}), ...);
}

template <int M, int Q, class LB, int... K>
RNS_TD void lazy_outputs(uint32_t (&v)[M], std::integer_sequence<int, K...>) {
  constexpr int LOG = ilog2(M);
  const uint32_t t[M] = {lazy_reduce<Q, LB::plan.ofold[K][2]>(lazy_reduce<Q, LB::plan.ofold[K][1]>(
      lazy_reduce<Q, LB::plan.ofold[K][0]>(v[bitrev(K, LOG)])))...};
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] = t[k];
}

// In-register transform V[k] = sum_n v[n] w^(n k), w = psi^(+-2048/M)
// (DIR 0: +, 1: -), radix-2 decimation in frequency with the bit-reversed
// output order undone by renaming registers, under the lazy bounds above.
template <int M, int DIR, int Q, int IB0, int IB, int OB0, int OB>
RNS_TD void dft(uint32_t (&v)[M]) {
  using LB = LazyBounds<M, IB0, IB, OB0, OB>;
  lazy_stages<M, DIR, Q, LB>(v, std::make_integer_sequence<int, ilog2(M)>{});
  lazy_outputs<M, Q, LB>(v, std::make_integer_sequence<int, M>{});
}

RNS_TD uint4 load_tw(const uint4 *p) {
#ifdef __CUDA_ARCH__
  return __ldg(p);
#else
  return *p;
#endif
}

// Pre-twist of a phase-A input u (any 32-bit value) at row n2: [0, 2p).
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
  dft<16, 0, 0, 2, 2, 16, 16>(v[0]);  // every output is twisted (a Shoup product)
  dft<16, 0, 1, 2, 2, 16, 16>(v[1]);
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
RNS_TD void fwd_phase_c1(uint2 *buf, int wg, int lane, const uint4 *c1tab) {
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
    dft<8, 0, 0, 2, 2, 2, 16>(u0);  // outputs c >= 1 are multiplied below; c = 0 feeds C2
    dft<8, 0, 1, 2, 2, 2, 16>(u1);
    row[a] = make_uint2(u0[0], u1[0]);
#pragma unroll
    for (int c = 1; c < 8; ++c) {
      const uint4 T = load_tw(c1tab + a * 8 + c);  // warp-uniform: one broadcast load
      row[c * 8 + a] = make_uint2(shoup<0>(u0[c], T.x, T.y), shoup<1>(u1[c], T.z, T.w));
    }
  }
}

// Phase C2: thread (k2, c) = (t & 15, t >> 4), both polynomials.  Outputs
// lie below 16p (the key products accept any 32-bit value).
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
    dft<8, 0, 0, 2, 2, 16, 16>(X[0][Pp]);  // outputs feed products: any bound
    dft<8, 0, 1, 2, 2, 16, 16>(X[1][Pp]);
  }
}

// ------------------------------------------------------------ inverse ---
// tw_inv: psi^(-n1 (2 k2 + 1)) / 1024 at [k2 * 64 + n1].
//
// Inputs of the inverse lie below kInvIn p: the transform-domain sums of a
// CMux step are three Montgomery-reduced level sums, each below 3p (two
// products of an input below 16p and a key below p sum below 32 p^2, and a
// Montgomery reduction of x < 32 p^2 lies below 32 p^2 / 2^32 + p < 3p).
constexpr int kInvIn = 9;

RNS_TD void inv_phase_c2(uint32_t (&X)[2][2][8], uint2 *buf, int t) {
  const int k2 = t & 15, c = t >> 4;
#pragma unroll
  for (int Pp = 0; Pp < 2; ++Pp) {
    dft<8, 1, 0, kInvIn, kInvIn, 16, 16>(X[0][Pp]);
    dft<8, 1, 1, kInvIn, kInvIn, 16, 16>(X[1][Pp]);
    uint2 *row = buf + (Pp * 16 + k2) * kRow + c * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) row[a] = make_uint2(X[0][Pp][a], X[1][Pp][a]);
  }
}

RNS_TD void inv_phase_c1(uint2 *buf, int wg, int lane, const uint4 *c1tab) {
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
      const uint4 T = load_tw(c1tab + a * 8 + c);
      u0[c] = shoup<0>(x.x, T.x, T.y);
      u1[c] = shoup<1>(x.y, T.z, T.w);
    }
    dft<8, 1, 0, 16, 2, 16, 16>(u0);  // phase A multiplies every output
    dft<8, 1, 1, 16, 2, 16, 16>(u1);
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
  dft<16, 1, 0, 2, 2, 4, 16>(v[0]);  // outputs n2 >= 1 are multiplied below; n2 = 0
  dft<16, 1, 1, 2, 2, 4, 16>(v[1]);  // goes to the reconstruction, which takes [0, 4p)
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
// each, below 16p.  tw: the factor table (kTwEntries entries).
__device__ __forceinline__ void forward(uint32_t (&v)[2][16], uint32_t (&X)[2][2][8], uint2 *buf,
                                        int t, int bar, int nthr, const uint4 *tw) {
  named_bar(bar, nthr);  // the buffer is free
  fwd_phase_a(v, buf, t, tw);
  named_bar(bar, nthr);
  fwd_phase_c1(buf, t >> 5, t & 31, tw + kTwC1Fwd);
  named_bar(bar, nthr);
  fwd_phase_c2(X, buf, t);
}

// Inverse transform: X (clobbered, values below kInvIn p) holds this thread's
// positions of both polynomials; v receives x_Pp[n1 + 64 n2].
__device__ __forceinline__ void inverse(uint32_t (&X)[2][2][8], uint32_t (&v)[2][16], uint2 *buf,
                                        int t, int bar, int nthr, const uint4 *tw) {
  named_bar(bar, nthr);
  inv_phase_c2(X, buf, t);
  named_bar(bar, nthr);
  inv_phase_c1(buf, t >> 5, t & 31, tw + kTwC1Inv);
  named_bar(bar, nthr);
  inv_phase_a(v, buf, t, tw + kTwInv);
}
#endif

}  // namespace rns
