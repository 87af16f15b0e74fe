// 1024-point negacyclic number-theoretic transform over F_p (p = 2^64 - 2^32
// + 1), applied to two polynomials at once by 128 threads.
//
// Used for the exact products of the blind rotation's external product
// (digit polynomial x bootstrapping-key polynomial, each CMux step).  The
// transform evaluates x(X) at the odd powers psi^(2k+1) of a primitive
// 2048-th root of unity psi chosen with psi^32 = 8, so that the pointwise
// product of two transforms is the transform of the product mod X^1024 + 1.
//
// Four-step split n = n1 + 64 n2, k = k2 + 16 k1:
//   A  : for each n1, a negacyclic 16-point transform over n2 with root
//        psi^64 = 2^6 (twiddles are powers of two), then the twist
//        psi^((2 k2 + 1) n1) (the only general multiplications);
//   C1 : the 64-point cyclic transform over n1 (root psi^32 = 8) as 8 x 8:
//        8-point transforms over b (n1 = a + 8 b, root 2^24), then the
//        power-of-two twiddle 8^(a c);
//   C2 : 8-point transforms over a, giving k1 = c + 8 d.
// Thread t (0..127 within its group) ends owning the same eight transform
// positions k = (t & 15) + 16 ((t >> 4) + 8 d), d = 0..7, of both
// polynomials, so pointwise work needs no data exchange.  Data moves between
// phases through a shared buffer of [2][16][65] uint64 (the padding makes
// every access of a warp conflict-free).  The inverse runs the phases
// backwards with inverse roots; the 1/1024 scale is folded into its twist.
#pragma once

#include "gl_field.cuh"

namespace ntt {

constexpr int kRow = 65;                 // padded row of the transpose buffer
constexpr int kBufWords = 2 * 16 * kRow; // uint64 words per 128-thread group

// Barrier `id` over `count` threads (all groups of a block share one barrier
// so that every warp of the block runs the same code region at a time).
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

__host__ __device__ constexpr int bitrev(int k, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1) << (bits - 1 - i);
  return r;
}

__host__ __device__ constexpr int ilog2(int m) { return m <= 1 ? 0 : 1 + ilog2(m >> 1); }

// In-register transform V[k] = sum_n v[n] w^(n k), w = 2^W a primitive M-th
// root of unity (W * M = 0 mod 192).  Radix-2 decimation in frequency; the
// bit-reversed output order is undone by renaming registers.
template <int M, int W>
__device__ __forceinline__ void dft(uint64_t (&v)[M]) {
  constexpr int LOG = ilog2(M);
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
    const int len = M >> (st + 1);
#pragma unroll
    for (int j0 = 0; j0 < M; j0 += 2 * len) {
#pragma unroll
      for (int i = 0; i < len; ++i) {
        const uint64_t a = v[j0 + i], b = v[j0 + i + len];
        v[j0 + i] = gl::add(a, b);
        v[j0 + i + len] = gl::mul_pow2(gl::sub(a, b), (W * i * (M / (2 * len))) % 192);
      }
    }
  }
  uint64_t t[M];
#pragma unroll
  for (int k = 0; k < M; ++k) t[k] = v[bitrev(k, LOG)];
#pragma unroll
  for (int k = 0; k < M; ++k) v[k] = t[k];
}

// ------------------------------------------------------------ forward ---

// Phase A: thread (P, n1) = (t >> 6, t & 63) holds v[n2] = x_P[n1 + 64 n2]
// already multiplied by the negacyclic pre-twist 2^(6 n2).
__device__ __forceinline__ void fwd_phase_a(uint64_t (&v)[16], uint64_t *buf, int t,
                                            const uint64_t *__restrict__ tw_fwd) {
  const int P = t >> 6, n1 = t & 63;
  dft<16, 12>(v);
  uint64_t *col = buf + P * 16 * kRow + n1;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) col[k2 * kRow] = gl::mul(v[k2], __ldg(tw_fwd + k2 * 64 + n1));
}

// Phase C1 for warp wg of the group: lane -> (P, k2) = (lane >> 4, lane & 15),
// a in {2 wg, 2 wg + 1}.  a is warp-uniform, so the shift of the twiddle
// 8^(a c) is the same across the warp (uniform branches, one code copy).
// The thread reads positions a + 8 b and writes positions 8 c + a of its row:
// the same eight positions, touched by no other thread, so the transform is
// done in place one a at a time without a barrier in between.
__device__ __forceinline__ void fwd_phase_c1(uint64_t *buf, int wg, int lane) {
  uint64_t *row = buf + ((lane >> 4) * 16 + (lane & 15)) * kRow;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int a = 2 * wg + j;
    uint64_t u[8];
#pragma unroll
    for (int b = 0; b < 8; ++b) u[b] = row[a + 8 * b];
    dft<8, 24>(u);
#pragma unroll
    for (int c = 0; c < 8; ++c) row[c * 8 + a] = gl::mul_pow2_uniform(u[c], (3 * a * c) % 192);
  }
}

// Phase C2: thread (k2, c) = (t & 15, t >> 4) for both polynomials.
__device__ __forceinline__ void fwd_phase_c2(uint64_t (&X)[2][8], const uint64_t *buf, int t) {
  const int k2 = t & 15, c = t >> 4;
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    const uint64_t *row = buf + (P * 16 + k2) * kRow + c * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) X[P][a] = row[a];
    dft<8, 24>(X[P]);
  }
}

// Forward transform of two polynomials; v holds the phase-A inputs of this
// thread, already pre-twisted (clobbered); X receives the eight positions
// of each polynomial.
__device__ __forceinline__ void forward_pretwisted(uint64_t (&v)[16], uint64_t (&X)[2][8],
                                                   uint64_t *buf, int t, int bar, int nthr,
                                                   const uint64_t *__restrict__ tw_fwd) {
  named_bar(bar, nthr);  // the buffer is free
  fwd_phase_a(v, buf, t, tw_fwd);
  named_bar(bar, nthr);
  fwd_phase_c1(buf, t >> 5, t & 31);
  named_bar(bar, nthr);
  fwd_phase_c2(X, buf, t);
}

// Forward transform of untwisted inputs v[n2] = x_P[n1 + 64 n2].
__device__ __forceinline__ void forward(uint64_t (&v)[16], uint64_t (&X)[2][8], uint64_t *buf,
                                        int t, int bar, int nthr,
                                        const uint64_t *__restrict__ tw_fwd) {
#pragma unroll
  for (int n2 = 1; n2 < 16; ++n2) v[n2] = gl::mul_pow2(v[n2], 6 * n2);
  forward_pretwisted(v, X, buf, t, bar, nthr, tw_fwd);
}

// ------------------------------------------------------------ inverse ---

__device__ __forceinline__ void inv_phase_c2(uint64_t (&X)[2][8], uint64_t *buf, int t) {
  const int k2 = t & 15, c = t >> 4;
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    dft<8, 168>(X[P]);
    uint64_t *row = buf + (P * 16 + k2) * kRow + c * 8;
#pragma unroll
    for (int a = 0; a < 8; ++a) row[a] = X[P][a];
  }
}

__device__ __forceinline__ void inv_phase_c1(uint64_t *buf, int wg, int lane) {
  uint64_t *row = buf + ((lane >> 4) * 16 + (lane & 15)) * kRow;
#pragma unroll 1
  for (int j = 0; j < 2; ++j) {
    const int a = 2 * wg + j;
    uint64_t u[8];
#pragma unroll
    for (int c = 0; c < 8; ++c)
      u[c] = gl::mul_pow2_uniform(row[c * 8 + a], (192 - (3 * a * c) % 192) % 192);
    dft<8, 168>(u);
#pragma unroll
    for (int b = 0; b < 8; ++b) row[a + 8 * b] = u[b];
  }
}

__device__ __forceinline__ void inv_phase_a(uint64_t (&v)[16], const uint64_t *buf, int t,
                                            const uint64_t *__restrict__ tw_inv) {
  const int P = t >> 6, n1 = t & 63;
  const uint64_t *col = buf + P * 16 * kRow + n1;
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) v[k2] = gl::mul(col[k2 * kRow], __ldg(tw_inv + k2 * 64 + n1));
  dft<16, 180>(v);
#pragma unroll
  for (int n2 = 1; n2 < 16; ++n2) v[n2] = gl::mul_pow2(v[n2], 192 - 6 * n2);
}

// Inverse transform: X (clobbered) holds this thread's positions of both
// polynomials; v receives x_P[n1 + 64 n2] for (P, n1) = (t >> 6, t & 63).
__device__ __forceinline__ void inverse(uint64_t (&X)[2][8], uint64_t (&v)[16], uint64_t *buf,
                                        int t, int bar, int nthr,
                                        const uint64_t *__restrict__ tw_inv) {
  named_bar(bar, nthr);
  inv_phase_c2(X, buf, t);
  named_bar(bar, nthr);
  inv_phase_c1(buf, t >> 5, t & 31);
  named_bar(bar, nthr);
  inv_phase_a(v, buf, t, tw_inv);
}

}  // namespace ntt
