// Blind rotation with the external product on the 5th-generation tensor
// cores (tcgen05): the Toeplitz form of the CMux step (hot-path step a3;
// TFHE's blind rotation, §3 "TFHE Library").
//
// One CMux step of a batch of gates adds to each accumulator half o
//   ACC_o[n] += sum_r sum_j digit_r[j] * bt_{r,o}[n - j]   (mod 2^32),
//   bt[s] = BSK_i[r][o][s] (s >= 0), -BSK_i[r][o][s + N] (s < 0)   (X^N = -1),
// over the six digit polynomials r = c*3 + p (accumulator half c, gadget
// level p).  For the whole batch that is one matrix product
//   [gates x 6N digits] x [6N x 2N] blocks of negacyclic Toeplitz matrices.
// With the digit coefficients reversed (k = N - 1 - j) every block is a
// Hankel matrix, f(n + k) with f(s) = bt[s - (N - 1)], so an 8 x 8 core
// matrix of the MMA operand depends only on (n + k) / 8: the key is stored
// once as the sequence of 255 core matrices CM_q[r][c] = f(8q + r + c), and
// the operand descriptor walks it with equal strides (LBO = SBO = 128 bytes)
// along both dimensions; nothing is expanded to N x N.
//
// Exactness on fp16 x fp16 -> fp32 MMAs: key words are split into four
// balanced byte limbs (|limb| <= 128) and digits (|d| <= 512) into two
// balanced 5-bit limbs (|limb| <= 16), so every accumulator sums 6N = 6144
// products of magnitude <= 2^11 and stays an exact integer below 2^24:
//   delta = sum_{a < 4, b < 2} 2^(8a + 5b) S_{a,b}   (mod 2^32).
// (Integer MMAs, kind::i8, do not exist on sm_103a; fp16 limbs carry the
// same eight limb products.)
//
// Per CMux step two launches: the digit kernel writes the gadget digits of
// X^abar_i ACC - ACC for every gate, already in the MMA operand layout; the
// MMA kernel computes, per CTA, a tile of 128 gates (M, TMEM lanes) x 128
// output coefficients (N) with the four key limbs in four accumulators (the
// whole 512-column TMEM), in two sweeps over K (low digit limb, then high),
// each followed by an epilogue that recombines the limbs and adds into ACC.
// K streams in chunks of 256 through a two-slot ring: a chunk boundary (the
// barrier wait and commit) costs about as much as 7 MMAs, so wide chunks win.
// Every wait is bounded (2 s on %globaltimer, then an error flag and an
// orderly exit).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "bounded_wait.cuh"
#include "ce_internal.h"
#include "launch.h"

namespace ce {

namespace {

constexpr int kTtM = 128;                             // gates per tile (MMA M)
constexpr int kTtN = 128;                             // output coefficients per tile (MMA N)
constexpr int kTtKC = 256;                            // K per pipeline chunk
constexpr int kTtRows = 2 * kGadgetL;                 // six digit polynomials
constexpr int kTtChunks = kTtRows * kRingN / kTtKC;   // 24 chunks per sweep
constexpr int kTtChunksPerRow = kRingN / kTtKC;       // 4
constexpr int kTtCoefTiles = 2 * kRingN / kTtN;       // 16
constexpr int kTtLimbs = 4;                           // key limbs
constexpr int kTtQ = 2 * kRingN / 8 - 1;              // 255 core matrices per sequence
constexpr int kTtSlots = 2;
constexpr int kTtABytes = kTtM * kTtKC * 2;           // 65,536: digit operand of a chunk
constexpr int kTtBBlocks = kTtN / 8 + kTtKC / 8 - 1;  // 47 core matrices per key limb
constexpr int kTtBLimbBytes = kTtBBlocks * 128;       // 6,016
constexpr int kTtStage = kTtABytes + kTtLimbs * kTtBLimbBytes;  // 89,600
constexpr int kTtASbo = (kTtKC / 8) * 128;            // 4,096: 8-row groups of the digits
constexpr uint32_t kTtTmemCols = 512;
constexpr uint32_t kDecompOffset = 0x80200802u;       // as in the transform path

static_assert(kTtLimbs * kTtN <= int(kTtTmemCols), "four accumulators fit in TMEM");
static_assert(kTtStage % 128 == 0 && kTtBLimbBytes % 16 == 0, "bulk copies stay 16-byte aligned");
// The highest core matrix a chunk reads: q0 + 46 with q0 = (n0 + k0) / 8.
static_assert((kRingN - kTtN + kRingN - kTtKC) / 8 + kTtBBlocks - 1 < kTtQ, "Hankel range");

struct TtSmem {
  static constexpr size_t kStages = size_t(kTtSlots) * kTtStage;
  static constexpr size_t kBars = size_t(2 * kTtSlots + 2) * 8;
  static constexpr size_t kTotal = kStages + kBars + 32 + 128;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return smem_addr(p); }

// fp16 bit pattern of an integer with |x| <= 2048 (the conversion is exact).
__device__ __forceinline__ uint16_t fp16_of_int(int x) { return __half_as_ushort(__int2half_rn(x)); }

// Balanced limb a of x (x = sum_a 2^(8a) limb_a mod 2^32, limb in [-128, 127]).
__device__ __forceinline__ void byte_limbs(uint32_t x, int (&l)[kTtLimbs]) {
#pragma unroll
  for (int a = 0; a < kTtLimbs; ++a) {
    l[a] = int((x + 128u) & 255u) - 128;
    x = (x - uint32_t(l[a])) >> 8;
  }
}

// Shared-memory matrix descriptor (no swizzle, version 1 at bit 46).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(lbo >> 4) << 16) |
         (uint64_t(sbo >> 4) << 32) | (uint64_t(1) << 46);
}

// kind::f16 instruction descriptor: fp32 accumulator, fp16 A and B, both
// K-major, N = 128, M = 128.
constexpr uint32_t kTtIdesc = (1u << 4) | (uint32_t(kTtN >> 3) << 17) | (uint32_t(kTtM >> 4) << 24);

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// ------------------------------------------------------------ key layout ---
// Admission of the tensor form: coefficient key [i][r][o][N] (uint32) to the
// Hankel limb sequences [i][r][o][limb][q < 255][8 x 8] (fp16).  Block (i, r, o).
__global__ void __launch_bounds__(256) bsk_to_hankel_kernel(const uint32_t *__restrict__ bsk,
                                                            uint16_t *__restrict__ hankel) {
  __shared__ int8_t lim[kTtLimbs][2 * kRingN];
  const uint32_t *b = bsk + size_t(blockIdx.x) * kRingN;
  for (int s = threadIdx.x; s < 2 * kRingN - 1; s += blockDim.x) {
    // f(s) = bt[s - (N - 1)]
    const int j = s - (kRingN - 1);
    const uint32_t f = j >= 0 ? b[j] : 0u - b[j + kRingN];
    int l[kTtLimbs];
    byte_limbs(f, l);
#pragma unroll
    for (int a = 0; a < kTtLimbs; ++a) lim[a][s] = int8_t(l[a]);
  }
  if (threadIdx.x < kTtLimbs) lim[threadIdx.x][2 * kRingN - 1] = 0;
  __syncthreads();
  uint4 *dst = reinterpret_cast<uint4 *>(hankel + size_t(blockIdx.x) * kTtLimbs * kTtQ * 64);
  // one 16-byte row (8 halves) of core matrix q of limb a per item
  for (int it = threadIdx.x; it < kTtLimbs * kTtQ * 8; it += blockDim.x) {
    const int a = it / (kTtQ * 8), q = (it / 8) % kTtQ, r = it % 8;
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      const int s = 8 * q + r + c;
      w[c / 2] = uint32_t(fp16_of_int(lim[a][s])) | (uint32_t(fp16_of_int(lim[a][s + 1])) << 16);
    }
    dst[it] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// ------------------------------------------------------------------ init ---
// ACC = (0, X^(-bbar) v), v = mu * sum_j X^j, mu = +1/8.  Block per job.
__global__ void __launch_bounds__(256) tt_init_kernel(const uint16_t *__restrict__ abar,
                                                      uint32_t *__restrict__ acc) {
  const int g = blockIdx.x;
  const int bbar = abar[size_t(g) * kAbarStride + kLweN];
  const int k = (2 * kRingN - bbar) & (2 * kRingN - 1);
  uint32_t *A = acc + size_t(g) * 2 * kRingN;
  for (int j = threadIdx.x; j < kRingN; j += blockDim.x) {
    A[j] = 0;
    const bool hi = k < kRingN ? (j >= k) : (j < k - kRingN);
    A[kRingN + j] = hi ? kMuEighth : 0u - kMuEighth;
  }
}

// ---------------------------------------------------------------- digits ---
// Block: 8 gates (one 8-row group of the digit operand), 256 threads.  Digit
// p of coefficient n of half c of D = X^abar_i ACC - ACC goes to K index
// (c*3 + p)*N + (N - 1 - n), split into a low and a high 5-bit limb; limb b
// of gate tile T, chunk ch is one contiguous 64 KB block of 16 x 32 core
// matrices (gates x K).  Gates beyond n_jobs get zero digits.
__global__ void __launch_bounds__(256) tt_digits_kernel(const uint32_t *__restrict__ acc,
                                                        const uint16_t *__restrict__ abar,
                                                        int step, int n_jobs, int n_tiles,
                                                        uint16_t *__restrict__ digits) {
  extern __shared__ __align__(16) uint32_t s_acc[];  // [8][2N]
  __shared__ int s_rot[8];
  const int g0 = blockIdx.x * 8;
  for (int idx = threadIdx.x; idx < 8 * (2 * kRingN / 4); idx += blockDim.x) {
    const int gi = idx / (2 * kRingN / 4), w4 = idx % (2 * kRingN / 4);
    const int g = g0 + gi;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (g < n_jobs) v = reinterpret_cast<const uint4 *>(acc + size_t(g) * 2 * kRingN)[w4];
    reinterpret_cast<uint4 *>(s_acc)[idx] = v;
  }
  if (threadIdx.x < 8) {
    const int g = g0 + threadIdx.x;
    s_rot[threadIdx.x] = g < n_jobs ? int(abar[size_t(g) * kAbarStride + step]) : 0;
  }
  __syncthreads();
  const int T = g0 / kTtM, R = (g0 % kTtM) / 8;
  for (int item = threadIdx.x; item < 2 * (kRingN / 8) * 8; item += blockDim.x) {
    const int gi = item & 7, k8 = (item >> 3) & (kRingN / 8 - 1), c = item >> 10;
    const int rot = s_rot[gi];
    const int kk = rot & (kRingN - 1);
    const uint32_t flip = rot >= kRingN ? 0xFFFFFFFFu : 0u;
    const uint32_t *src = s_acc + gi * 2 * kRingN + c * kRingN;
    uint32_t lo[kGadgetL][4], hi[kGadgetL][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int n = kRingN - 1 - (8 * k8 + e);
      const int s = n - kk;
      uint32_t r = s >= 0 ? src[s] : 0u - src[s + kRingN];
      r = (r ^ flip) - flip;  // X^N = -1
      const uint32_t w = r - src[n] + kDecompOffset;
#pragma unroll
      for (int p = 0; p < kGadgetL; ++p) {
        const int d = int((w >> (22 - 10 * p)) & 1023u) - 512;
        const int l = ((d + 16) & 31) - 16;
        const int h = (d - l) >> 5;
        const uint32_t lb = fp16_of_int(l), hb = fp16_of_int(h);
        if (e & 1) {
          lo[p][e / 2] |= lb << 16;
          hi[p][e / 2] |= hb << 16;
        } else {
          lo[p][e / 2] = lb;
          hi[p][e / 2] = hb;
        }
      }
    }
#pragma unroll
    for (int p = 0; p < kGadgetL; ++p) {
      constexpr int kCm = kTtKC / 8;  // core matrices along K in a chunk
      const int ch = (c * kGadgetL + p) * kTtChunksPerRow + k8 / kCm, C = k8 % kCm;
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const size_t off =
            ((((size_t(b) * n_tiles + T) * kTtChunks + ch) * (kTtM / 8) + R) * kCm + C) * 64 +
            gi * 8;
        const uint32_t(&v)[4] = b ? hi[p] : lo[p];
        *reinterpret_cast<uint4 *>(digits + off) = make_uint4(v[0], v[1], v[2], v[3]);
      }
    }
  }
}

// ------------------------------------------------------------------- MMA ---
// Stream-K schedule.  The step's work is U = tiles x 16 coefficient tiles x
// 48 units (2 sweeps x 24 chunks of K), ordered (gate tile, coefficient
// tile, sweep, chunk); CTA b of the grid takes the contiguous range
// [b U / G, (b + 1) U / G).  A piece is a maximal run of one (tile, sweep)
// inside that range; each piece ends with an epilogue that adds its partial
// sums into ACC, with atomics unless the CTA owns both sweeps of the tile
// (exact mod 2^32 either way).  Every CTA gets the same amount of work up to
// one unit, whatever the batch size: no partial last wave.
constexpr int kTtUnitsPerSweep = kTtChunks;                  // 24
constexpr int kTtUnitsPerTile = 2 * kTtUnitsPerSweep;        // 48

struct TtPiece {
  int tile, sweep, first, count;  // tile = gate tile * 16 + coefficient tile
  bool shared;                    // another CTA adds into the same outputs
};

// Piece p of the range [u0, u1) (p = 0, 1, ...; count 0 past the end).
__device__ __forceinline__ TtPiece tt_piece(long long u0, long long u1, int p) {
  TtPiece q{0, 0, 0, 0, false};
  const long long s0 = u0 / kTtUnitsPerSweep;
  const long long s = s0 + p;  // global sweep-run index
  const long long lo = s * kTtUnitsPerSweep > u0 ? s * kTtUnitsPerSweep : u0;
  long long hi = (s + 1) * kTtUnitsPerSweep;
  if (hi > u1) hi = u1;
  if (hi <= lo) return q;
  q.tile = int(s / 2);
  q.sweep = int(s % 2);
  q.first = int(lo % kTtUnitsPerSweep);
  q.count = int(hi - lo);
  const long long t0 = (long long)q.tile * kTtUnitsPerTile;
  q.shared = !(u0 <= t0 && t0 + kTtUnitsPerTile <= u1);
  return q;
}

// grid (G), 192 threads: warps 0-3 epilogue (TMEM lane quarters), warp 4
// lane 0 copies, warp 5 lane 0 issues MMAs.  hankel_i: the step's key
// sequences [r][o][limb][q][64].
__global__ void __launch_bounds__(192, 1) tt_mma_kernel(const uint16_t *__restrict__ digits,
                                                        const uint16_t *__restrict__ hankel_i,
                                                        uint32_t *__restrict__ acc, int n_jobs,
                                                        int n_tiles, int *__restrict__ err) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + TtSmem::kStages);
  uint64_t *empty = full + kTtSlots;
  uint64_t *acc_full = empty + kTtSlots;
  uint64_t *tmem_free = acc_full + 1;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tmem_free + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *n_issued = abort + 1;
  volatile int *n_landed = abort + 2;
  volatile int *n_committed = abort + 3;

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const long long U = (long long)n_tiles * kTtCoefTiles * kTtUnitsPerTile;
  const long long u0 = U * blockIdx.x / gridDim.x, u1 = U * (blockIdx.x + 1) / gridDim.x;
  const int total = int(u1 - u0);

  if (t == 0) {
    for (int s = 0; s < kTtSlots; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + s)) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(acc_full)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(tmem_free)) : "memory");
    *abort = 0;
    *n_issued = 0;
    *n_landed = 0;
    *n_committed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTtTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 4 && lane == 0) {
    // Producer: unit c of the range; digits of limb `sweep` (chunk ch of
    // gate tile T), key sequences of digit row r = ch / 4 from
    // q0 = (n0 + k0) / 8.
    int c = 0;
    for (int p = 0; c < total; ++p) {
      const TtPiece pc = tt_piece(u0, u1, p);
      const int T = pc.tile / kTtCoefTiles, ct = pc.tile % kTtCoefTiles;
      const int o = ct / (kRingN / kTtN), n0 = (ct % (kRingN / kTtN)) * kTtN;
      for (int i = 0; i < pc.count; ++i, ++c) {
        const int slot = c % kTtSlots;
        if (c >= kTtSlots &&
            !bounded_wait(smem_u32(empty + slot), uint32_t(c / kTtSlots - 1) & 1u, abort, err))
          break;
        if (*abort) break;
        const int ch = pc.first + i;
        const int r = ch / kTtChunksPerRow, k0 = (ch % kTtChunksPerRow) * kTtKC;
        const int q0 = (n0 + k0) / 8;
        uint8_t *st = smem + size_t(slot) * kTtStage;
        const uint32_t bar = smem_u32(full + slot);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"(uint32_t(kTtStage))
                     : "memory");
        bulk_copy(st,
                  digits + ((size_t(pc.sweep) * n_tiles + T) * kTtChunks + ch) * (kTtABytes / 2),
                  kTtABytes, bar);
#pragma unroll
        for (int a = 0; a < kTtLimbs; ++a)
          bulk_copy(st + kTtABytes + a * kTtBLimbBytes,
                    hankel_i + ((size_t(r * 2 + o) * kTtLimbs + a) * kTtQ + q0) * 64,
                    kTtBLimbBytes, bar);
        *n_issued = c + 1;
      }
      if (*abort) break;
    }
  } else if (warp == 5 && lane == 0) {
    // MMA issuer: per unit 16 K-steps x 4 key limbs; the accumulators restart
    // at each piece, whose first MMA waits until the epilogue has read the
    // previous piece out of TMEM.
    int c = 0;
    bool ok = true;
    for (int p = 0; ok && c < total; ++p) {
      const TtPiece pc = tt_piece(u0, u1, p);
      if (p > 0) {
        if (!bounded_wait(smem_u32(tmem_free), uint32_t(p - 1) & 1u, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
      for (int i = 0; i < pc.count; ++i, ++c) {
        const int slot = c % kTtSlots;
        if (!bounded_wait(smem_u32(full + slot), uint32_t(c / kTtSlots) & 1u, abort, err)) {
          ok = false;
          break;
        }
        *n_landed = c + 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(smem + size_t(slot) * kTtStage);
        const uint32_t b0 = a0 + kTtABytes;
#pragma unroll
        for (int s = 0; s < kTtKC / 16; ++s) {
          const uint64_t ad = smem_desc(a0 + s * 256, 128, kTtASbo);
          const uint32_t accum = (i != 0 || s != 0) ? 1u : 0u;
#pragma unroll
          for (int a = 0; a < kTtLimbs; ++a) {
            const uint64_t bd = smem_desc(b0 + a * kTtBLimbBytes + s * 256, 128, 128);
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                    tmem + uint32_t(a * kTtN)),
                "l"(ad), "l"(bd), "r"(kTtIdesc), "r"(accum)
                : "memory");
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(empty + slot))
            : "memory");
        if (i + 1 == pc.count)
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_u32(acc_full))
              : "memory");
        *n_committed = c + 1;
      }
    }
  } else if (warp < 4) {
    // Epilogue: warp w holds gates 32 w .. 32 w + 31 of the piece's tile.
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    int c = 0;
    for (int p = 0; c < total; ++p) {
      const TtPiece pc = tt_piece(u0, u1, p);
      c += pc.count;
      const int T = pc.tile / kTtCoefTiles, ct = pc.tile % kTtCoefTiles;
      const int o = ct / (kRingN / kTtN), n0 = (ct % (kRingN / kTtN)) * kTtN;
      const int g = T * kTtM + warp * 32 + lane;
      if (!bounded_wait(smem_u32(acc_full), uint32_t(p) & 1u, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int nb = 0; nb < kTtN / 16; ++nb) {
        uint32_t v[kTtLimbs][16];
#pragma unroll
        for (int a = 0; a < kTtLimbs; ++a) {
          const uint32_t addr = tmem + lane_base + uint32_t(a * kTtN + nb * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
              "%13,%14,%15}, [%16];"
              : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]),
                "=r"(v[a][5]), "=r"(v[a][6]), "=r"(v[a][7]), "=r"(v[a][8]), "=r"(v[a][9]),
                "=r"(v[a][10]), "=r"(v[a][11]), "=r"(v[a][12]), "=r"(v[a][13]), "=r"(v[a][14]),
                "=r"(v[a][15])
              : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (g >= n_jobs) continue;
        uint32_t d[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          uint32_t x = 0;
#pragma unroll
          for (int a = 0; a < kTtLimbs; ++a)
            x += uint32_t(__float2int_rn(__uint_as_float(v[a][j]))) << (8 * a);
          d[j] = x << (5 * pc.sweep);
        }
        uint32_t *dst = acc + size_t(g) * 2 * kRingN + o * kRingN + n0 + nb * 16;
        if (!pc.shared) {
          uint4 *d4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint4 y = d4[q];
            y.x += d[4 * q];
            y.y += d[4 * q + 1];
            y.z += d[4 * q + 2];
            y.w += d[4 * q + 3];
            d4[q] = y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) atomicAdd(dst + j, d[j]);
        }
      }
      if (c < total) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0)
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(tmem_free))
                       : "memory");
      }
    }
  }
  __syncthreads();
  if (warp == 5 && lane == 0 && *abort) {
    // Orderly exit after an expired wait: issued copies land and committed
    // MMAs finish before shared memory and TMEM are released.
    const int issued = *n_issued, landed = *n_landed, committed = *n_committed;
    for (int c = landed; c < issued; ++c)
      drain_wait(smem_u32(full + c % kTtSlots), uint32_t(c / kTtSlots) & 1u);
    if (committed > 0)
      drain_wait(smem_u32(empty + (committed - 1) % kTtSlots),
                 uint32_t((committed - 1) / kTtSlots) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTtTmemCols)
                 : "memory");
}

}  // namespace

size_t blind_rotate_tc_key_bytes() {
  return size_t(kLweN) * kTtRows * 2 * kTtLimbs * kTtQ * 64 * sizeof(uint16_t);
}

size_t blind_rotate_tc_digit_bytes(size_t n_jobs) {
  const size_t tiles = (n_jobs + kTtM - 1) / kTtM;
  return 2 * tiles * kTtChunks * size_t(kTtABytes);
}

cudaError_t launch_bsk_to_hankel(const uint32_t *bsk, uint16_t *hankel, cudaStream_t st) {
  bsk_to_hankel_kernel<<<kLweN * kTtRows * 2, 256, 0, st>>>(bsk, hankel);
  return cudaGetLastError();
}

// CTAs of a step's MMA launch: one per SM (a stream-K range each), fewer
// only when the step has fewer units of work than SMs.
int blind_rotate_tc_ctas(int sms, int n_jobs) {
  const long long units =
      (long long)((n_jobs + kTtM - 1) / kTtM) * kTtCoefTiles * kTtUnitsPerTile;
  return int(units < sms ? units : sms);
}

cudaError_t launch_blind_rotate_tc(const uint16_t *hankel, const uint16_t *abar, uint32_t *acc,
                                   int n_jobs, uint16_t *digits, int ctas, int *err,
                                   cudaStream_t st, int *launches, cudaEvent_t *mma_ev) {
  if (n_jobs <= 0) return cudaSuccess;
  if (ctas < 1 || ctas > blind_rotate_tc_ctas(1 << 30, n_jobs)) return cudaErrorInvalidValue;
  const int n_tiles = (n_jobs + kTtM - 1) / kTtM;
  const int dig_smem = 8 * 2 * kRingN * 4;  // 64 KB
  cudaError_t e = cudaFuncSetAttribute(tt_digits_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, dig_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tt_mma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(TtSmem::kTotal));
  if (e != cudaSuccess) return e;
  tt_init_kernel<<<n_jobs, 256, 0, st>>>(abar, acc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t step_words = size_t(kTtRows) * 2 * kTtLimbs * kTtQ * 64;

  for (int i = 0; i < kLweN; ++i) {
    tt_digits_kernel<<<n_tiles * (kTtM / 8), 256, dig_smem, st>>>(acc, abar, i, n_jobs, n_tiles,
                                                                  digits);
    if (mma_ev) cudaEventRecord(mma_ev[2 * i], st);
    tt_mma_kernel<<<ctas, 192, TtSmem::kTotal, st>>>(digits, hankel + size_t(i) * step_words,
                                                     acc, n_jobs, n_tiles, err);
    if (mma_ev) cudaEventRecord(mma_ev[2 * i + 1], st);
  }
  e = cudaGetLastError();
  if (launches) *launches += 1 + 2 * kLweN;
  return e;
}

}  // namespace ce
