// LWE key switching on the 5th-generation tensor cores (tcgen05), fused with
// sample extraction (hot-path steps a4 + a5; TFHE's key switch, §3 "TFHE
// Library").
//
// Key switching sums, for every output, one key-switching-key row per
// (j, q) selected by the base-4 digit d = digit_q(round16(a'_j)):
//   out = (0, b') - sum_{j, q : d != 0} KSK[j][q][d]   (mod 2^32).
// That is a matrix product: a one-hot matrix H[output][(j, d, q)] (1 where
// the digit of (j, q) equals d) times the key K[(j, d, q)][word].  The key
// words are split into three 11-bit limbs (fp16-exact); every product is a
// limb value and every fp32 sum has at most 1024 * 8 terms below 2^11, so it
// stays an exact integer below 2^24.  Hence
//   sum = S0 + 2^11 S1 + 2^22 S2 (mod 2^32),
// with S_b = H x K_b computed exactly by kind::f16 MMAs with fp32
// accumulation.
//
// Tile of one CTA: 128 output words (MMA M, TMEM lanes) x N outputs (MMA N,
// up to 160) x the three limbs (three accumulators of N columns, each
// starting on a multiple of 32 TMEM columns), over
// a range of stages; a stage covers two values of j (K = 2 x 3 x 8 = 48).
// Operands sit in shared memory in the no-swizzle K-major core-matrix layout
// (8 rows x 16 bytes per core matrix; LBO = 128 B between core matrices along
// K, SBO = 768 B between 8-row groups):
//   - the key limbs were rearranged at admission into that layout, one
//     contiguous 36 KB block per (word tile, stage), fetched by one bulk copy;
//   - a pre-pass extracts and rounds the coefficients into [j][output]
//     (coalesced); the one-hot operand is written by the CTA's threads from
//     them (three 16-byte stores per output and j), one stage read ahead.
// Warp roles: four builder warps write the one-hot operand of each stage
// into a ring of four slots and signal it on the slot's "ready" mbarrier;
// one control warp (one thread) issues the key-limb bulk copies (the slot's
// "full" mbarrier) and, once both operands of a stage are in, the stage's
// MMAs (3 K-steps x 3 limbs), committed to the slot's "empty" mbarrier,
// which releases the slot to the builders and to the next copy.  Builders
// run up to four stages ahead of the tensor cores; no CTA-wide barrier sits
// between stages.  The builder warps then read the accumulators from TMEM
// (epilogue).  Every wait is bounded (2 s on %globaltimer, then an error
// flag and an orderly exit).
#include <cuda_runtime.h>

#include <cstdint>

#include "bounded_wait.cuh"
#include "ce_internal.h"
#include "launch.h"

namespace ce {

namespace {

constexpr int kTcM = 128;                    // output words per tile
constexpr int kTcWordTiles = kKskRow / kTcM; // 4
constexpr int kTcJPerStage = 2;
constexpr int kTcK = kTcJPerStage * 3 * kKsT;  // 48
constexpr int kTcStages = kRingN / kTcJPerStage;  // 512
constexpr int kTcSlots = 4;
constexpr int kTcBuilders = 4;                       // builder / epilogue warps
constexpr int kTcThreads = 32 * (kTcBuilders + 1);   // + the control warp
constexpr int kTcNMax = 160;
constexpr int kTcLbo = 128;                  // bytes between K-adjacent core matrices
constexpr int kTcSbo = (kTcK / 8) * 128;     // 768: bytes between 8-row groups
constexpr int kTcPlaneBytes = kTcM * kTcK * 2;        // 12,288
constexpr int kTcABytes = 3 * kTcPlaneBytes;          // 36,864 per stage
constexpr int kTcBBytes = kTcNMax * kTcK * 2;         // 15,360 per stage
constexpr uint32_t kTcTmemCols = 512;

static_assert(kTcWordTiles * kTcM == kKskRow, "word tiles cover a padded row");
static_assert(3 * kTcNMax <= int(kTcTmemCols), "three accumulators fit in TMEM");

struct TcSmem {
  static constexpr size_t kA = size_t(kTcSlots) * kTcABytes;
  static constexpr size_t kB = size_t(kTcSlots) * kTcBBytes;
  static constexpr size_t kBars = 3 * kTcSlots * 8;
  static constexpr size_t kTotal = kA + kB + kBars + 16 + 128;  // + TMEM address, abort, alignment
};

// Byte offset of element (row r, k) of a K-major operand tile with 48 columns.
__host__ __device__ constexpr uint32_t cm_offset(int r, int k) {
  return uint32_t((r >> 3) * kTcSbo + (k >> 3) * kTcLbo + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return smem_addr(p); }
// Bounded waits of this kernel (bounded_wait.cuh).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort,
                                          int *err) {
  return bounded_wait(bar, parity, abort, err);
}
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) { drain_wait(bar, parity); }

// Shared-memory matrix descriptor: start address, LBO, SBO (all >> 4),
// descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return uint64_t((addr & 0x3FFFFu) >> 4) | (uint64_t(kTcLbo >> 4) << 16) |
         (uint64_t(kTcSbo >> 4) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | (uint32_t(n >> 3) << 17) | (uint32_t(kTcM >> 4) << 24);
}

__device__ __forceinline__ void issue_stage_copy(uint8_t *dst, uint32_t bar, const uint8_t *src) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(uint32_t(kTcABytes))
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(uint32_t(kTcABytes)), "r"(bar)
      : "memory");
}

// Accumulators of the job(s) of output o (1 or 2; MUX adds the second).
struct OutJobs {
  int j1, j2;
};
__device__ __forceinline__ OutJobs out_jobs(int mode, const GateOut *outs, int o) {
  if (mode == 0) return OutJobs{o, -1};
  if (mode == 1) return OutJobs{2 * o, 2 * o + 1};
  return OutJobs{outs[o].job1, outs[o].job2};
}

// ---------------------------------------------------------------- kernel ---
// grid (word tile, output tile, k split).  n_tile: outputs per tile (multiple
// of 16, <= 160); stages_per_cta: stages of K in one CTA.  With a K split the
// outputs were zeroed and partial sums are added atomically (exact mod 2^32).
__global__ void __launch_bounds__(kTcThreads, 1) keyswitch_tc_kernel(
    const uint32_t *__restrict__ acc, const uint16_t *__restrict__ hr, int ldh,
    const uint8_t *__restrict__ planes, const GateOut *__restrict__ outs,
    uint32_t *__restrict__ out, int n_out, int mode, int n_tile, int stages_per_cta,
    int *__restrict__ err) {
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *smem = smem_raw;
  uint8_t *sa = smem;
  uint8_t *sb = smem + TcSmem::kA;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + TcSmem::kA + TcSmem::kB);
  uint64_t *ready = full + kTcSlots;
  uint64_t *empty = ready + kTcSlots;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty + kTcSlots);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wt = blockIdx.x, o0 = blockIdx.y * n_tile, ks = blockIdx.z;
  const int s0 = ks * stages_per_cta;
  const int n_stages = stages_per_cta;
  const uint8_t *a_src = planes + (size_t(wt) * kTcStages + s0) * kTcABytes;

  if (t == 0) {
    for (int s = 0; s < kTcSlots; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + s)) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(ready + s)),
                   "r"(kTcBuilders)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(empty + s)) : "memory");
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTcTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc(n_tile);
  const int col_stride = (n_tile + 31) & ~31;  // TMEM columns per limb accumulator

  // The control thread's record of the pipeline: stages whose key copy was
  // issued, whose copy was seen complete, and whose MMAs were committed.
  const bool control = warp == kTcBuilders;
  int issued = 0, landed = 0, committed = 0;
  if (control && lane == 0) {
    for (int s = 0; s < kTcSlots && s < n_stages; ++s, ++issued)
      issue_stage_copy(sa + size_t(s) * kTcABytes, smem_u32(full + s),
                       a_src + size_t(s) * kTcABytes);
    for (int i = 0; i < n_stages && !*abort; ++i) {
      const int slot = i % kTcSlots;
      const uint32_t par = uint32_t(i / kTcSlots) & 1u;
      if (!mbar_wait(smem_u32(full + slot), par, abort, err)) break;
      ++landed;
      if (!mbar_wait(smem_u32(ready + slot), par, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sa + size_t(slot) * kTcABytes);
      const uint32_t b0 = smem_u32(sb + size_t(slot) * kTcBBytes);
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t bd = smem_desc(b0 + kk * 2 * kTcLbo);
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
          const uint64_t ad = smem_desc(a0 + pl * kTcPlaneBytes + kk * 2 * kTcLbo);
          const uint32_t accum = (i | kk) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                  tmem + uint32_t(pl * col_stride)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(empty + slot))
          : "memory");
      ++committed;
      // Refill the previous stage's key slot once its MMAs are done (this
      // stage's MMAs keep the tensor cores busy meanwhile).
      if (i >= 1) {
        const int ps = (i - 1) % kTcSlots;
        if (!mbar_wait(smem_u32(empty + ps), uint32_t((i - 1) / kTcSlots) & 1u, abort, err))
          break;
        const int next = i - 1 + kTcSlots;
        if (next < n_stages) {
          issue_stage_copy(sa + size_t(ps) * kTcABytes, smem_u32(full + ps),
                           a_src + size_t(next) * kTcABytes);
          ++issued;
        }
      }
    }
  } else if (!control) {
    // Rounded coefficients of this thread's items (item it: j' = it / n_tile,
    // output o0 + it % n_tile), loaded one stage ahead; 0xFFFFFFFF marks a
    // padding row (all-zero one-hot).
    constexpr int kItems = (2 * kTcNMax + 127) / 128;
    auto load_h = [&](int stage, uint32_t (&hv)[kItems]) {
#pragma unroll
      for (int u = 0; u < kItems; ++u) {
        const int it = t + 128 * u;
        hv[u] = 0xFFFFFFFFu;
        if (it < 2 * n_tile && stage < n_stages) {
          const int jj = it >= n_tile, ol = it - jj * n_tile, o = o0 + ol;
          if (o < n_out) hv[u] = hr[size_t((s0 + stage) * kTcJPerStage + jj) * ldh + o];
        }
      }
    };
    uint32_t h_cur[kItems], h_next[kItems];
    load_h(0, h_cur);
    for (int i = 0; i < n_stages; ++i) {
      const int slot = i % kTcSlots;
      load_h(i + 1, h_next);
      if (i >= kTcSlots) {  // the slot's previous one-hot tile is consumed
        bool ok = true;
        if (lane == 0)
          ok = mbar_wait(smem_u32(empty + slot), uint32_t((i - kTcSlots) / kTcSlots) & 1u, abort,
                         err);
        if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) break;
      }
      // One-hot operand of this stage: rows = outputs of the tile, K = (j', d, q).
      uint8_t *b = sb + size_t(slot) * kTcBBytes;
#pragma unroll
      for (int u = 0; u < kItems; ++u) {
        const int it = t + 128 * u;
        if (it >= 2 * n_tile) break;
        const int jj = it >= n_tile, ol = it - jj * n_tile;
        const uint32_t h = h_cur[u];
        const bool live = h != 0xFFFFFFFFu;
        uint8_t *row = b + (ol >> 3) * kTcSbo + (ol & 7) * 16 + jj * 3 * kTcLbo;
#pragma unroll
        for (int d = 1; d <= 3; ++d) {
          uint32_t w[4];
#pragma unroll
          for (int pq = 0; pq < 4; ++pq) {
            const uint32_t d0 = (h >> (14 - 2 * (2 * pq))) & 3u;
            const uint32_t d1 = (h >> (14 - 2 * (2 * pq + 1))) & 3u;
            const uint32_t lo = (live && d0 == uint32_t(d)) ? 0x3C00u : 0u;  // fp16 1.0
            const uint32_t hi = (live && d1 == uint32_t(d)) ? 0x3C00u : 0u;
            w[pq] = lo | (hi << 16);
          }
          *reinterpret_cast<uint4 *>(row + (d - 1) * kTcLbo) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
#pragma unroll
      for (int u = 0; u < kItems; ++u) h_cur[u] = h_next[u];
      // make the generic-proxy stores visible to the tensor cores, then one
      // arrival per warp
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(ready + slot))
                     : "memory");
    }
  }
  __syncthreads();
  if (control && lane == 0 && *abort) {
    // Orderly exit after an expired wait: let issued copies land and the
    // committed MMAs finish before shared memory and TMEM are released.
    for (int s = landed; s < issued; ++s)
      mbar_drain(smem_u32(full + s % kTcSlots), uint32_t(s / kTcSlots) & 1u);
    if (committed > 0)
      mbar_drain(smem_u32(empty + (committed - 1) % kTcSlots),
                 uint32_t((committed - 1) / kTcSlots) & 1u);
  }
  __syncthreads();
  // The last stage's release barrier completes when every MMA has finished
  // (one waiting lane per builder warp; the TMEM loads below need the whole
  // warp to agree).
  bool ok = !*abort && !control;
  if (ok && n_stages > 0) {
    const int last = n_stages - 1;
    if (lane == 0)
      ok = mbar_wait(smem_u32(empty + last % kTcSlots), uint32_t(last / kTcSlots) & 1u, abort,
                     err);
    ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // Warp w holds words 32 w .. 32 w + 31 of the tile (TMEM lanes).
    const int m = wt * kTcM + warp * 32 + lane;
    const uint32_t lane_base = uint32_t(warp * 32) << 16;
    for (int c0 = 0; c0 < n_tile; c0 += 16) {
      uint32_t r[3][16];
#pragma unroll
      for (int pl = 0; pl < 3; ++pl) {
        const uint32_t addr = tmem + lane_base + uint32_t(pl * col_stride + c0);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];"
            : "=r"(r[pl][0]), "=r"(r[pl][1]), "=r"(r[pl][2]), "=r"(r[pl][3]), "=r"(r[pl][4]),
              "=r"(r[pl][5]), "=r"(r[pl][6]), "=r"(r[pl][7]), "=r"(r[pl][8]), "=r"(r[pl][9]),
              "=r"(r[pl][10]), "=r"(r[pl][11]), "=r"(r[pl][12]), "=r"(r[pl][13]), "=r"(r[pl][14]),
              "=r"(r[pl][15])
            : "r"(addr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m >= kLweWords) continue;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int o = o0 + c0 + c;
        if (o >= n_out || c0 + c >= n_tile) continue;
        const uint32_t sum = __float2uint_rn(__uint_as_float(r[0][c])) +
                             (__float2uint_rn(__uint_as_float(r[1][c])) << 11) +
                             (__float2uint_rn(__uint_as_float(r[2][c])) << 22);
        uint32_t val = 0u - sum;
        const OutJobs jb = out_jobs(mode, outs, o);
        if (m == kLweN && ks == 0) {
          uint32_t bp = acc[size_t(jb.j1) * 2 * kRingN + kRingN];
          if (jb.j2 >= 0) bp += acc[size_t(jb.j2) * 2 * kRingN + kRingN] + kMuEighth;
          val += bp;
        }
        uint32_t *dst = mode == 2 ? out + size_t(outs[o].slot) * kSlotWords
                                  : out + size_t(o) * kLweWords;
        if (gridDim.z == 1)
          dst[m] = val;
        else
          atomicAdd(dst + m, val);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcTmemCols)
                 : "memory");
}

// Sample extraction + rounding, h[j][o] = round16(a'_j) of output o with
// a'_0 = A_0, a'_j = -A_{N-j} (A = the output's accumulator, or the sum of
// its two for a MUX), stored with outputs contiguous so that the key switch
// reads a stage's coefficients coalesced.  Block (32 outputs, 32 j): reads
// along j, writes along o through a shared-memory transpose.
__global__ void __launch_bounds__(256) ks_round_kernel(const uint32_t *__restrict__ acc,
                                                       const GateOut *__restrict__ outs, int mode,
                                                       int n_out, uint16_t *__restrict__ hr,
                                                       int ldh) {
  __shared__ uint16_t tile[32][33];
  const int o0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {
    const int o = o0 + r, j = j0 + tx;
    uint16_t h = 0;
    if (o < n_out) {
      const OutJobs jb = out_jobs(mode, outs, o);
      const uint32_t *A = acc + size_t(jb.j1) * 2 * kRingN;
      uint32_t a = (j == 0) ? A[0] : 0u - A[kRingN - j];
      if (jb.j2 >= 0) {
        const uint32_t *A2 = acc + size_t(jb.j2) * 2 * kRingN;
        a += (j == 0) ? A2[0] : 0u - A2[kRingN - j];
      }
      h = uint16_t((a + 0x8000u) >> 16);
    }
    tile[r][tx] = h;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, o = o0 + tx;
    if (o < n_out) hr[size_t(j) * ldh + o] = tile[tx][r];
  }
}

// Admission: the device key-switching key [j][q][d-1][512] (uint32) to the
// three fp16 limb planes, tiled [word tile][stage][limb][core-matrix tile].
// Block (word tile, stage); K within a stage is k = 24 j' + 8 (d - 1) + q,
// the order in which the one-hot operand is written.
__global__ void __launch_bounds__(256) ksk_to_planes_kernel(const uint32_t *__restrict__ ksk,
                                                            uint16_t *__restrict__ planes) {
  const int wt = blockIdx.x, s = blockIdx.y;
  uint8_t *blk = reinterpret_cast<uint8_t *>(planes) + (size_t(wt) * kTcStages + s) * kTcABytes;
  for (int idx = threadIdx.x; idx < kTcM * kTcK; idx += blockDim.x) {
    const int r = idx / kTcK, k = idx % kTcK;
    const int jj = k / 24, d = (k % 24) / 8 + 1, q = k % 8;
    const int j = s * kTcJPerStage + jj, m = wt * kTcM + r;
    const uint32_t v = ksk[((size_t(j) * kKsT + q) * 3 + (d - 1)) * kKskRow + m];
    const uint32_t limb[3] = {v & 0x7FFu, (v >> 11) & 0x7FFu, v >> 22};
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
      // Integers below 2^11 are exact in fp16: exponent 15 + e, mantissa below the leading one.
      const uint32_t x = limb[pl];
      uint16_t bits = 0;
      if (x) {
        const int e = 31 - __clz(x);
        bits = uint16_t(((15 + e) << 10) | ((x << (10 - e)) & 0x3FFu));
      }
      *reinterpret_cast<uint16_t *>(blk + pl * kTcPlaneBytes + cm_offset(r, k)) = bits;
    }
  }
}

}  // namespace

size_t keyswitch_tc_plane_bytes() { return size_t(kTcWordTiles) * kTcStages * kTcABytes; }

cudaError_t launch_ksk_to_planes(const uint32_t *ksk, uint16_t *planes, cudaStream_t st) {
  ksk_to_planes_kernel<<<dim3(kTcWordTiles, kTcStages), 256, 0, st>>>(ksk, planes);
  return cudaGetLastError();
}

void keyswitch_tc_shape(int sms, int n_out, int *n_tile, int *out_tiles, int *ksplit) {
  int tiles = (n_out + kTcNMax - 1) / kTcNMax;
  if (tiles < 1) tiles = 1;
  int n = (n_out + tiles - 1) / tiles;
  n = (n + 15) / 16 * 16;
  if (n < 16) n = 16;
  int k = 1;
  while (k < 64 && kTcWordTiles * tiles * k * 2 <= sms) k *= 2;
  *n_tile = n;
  *out_tiles = tiles;
  *ksplit = k;
}

cudaError_t launch_keyswitch_tc(const uint32_t *acc, const uint16_t *planes, const GateOut *outs,
                                uint32_t *out, int n_out, int mode, int n_tile, int out_tiles,
                                int ksplit, uint16_t *h, int ldh, int *err, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  if (n_tile < 16 || n_tile > kTcNMax || n_tile % 16 || ksplit < 1 || kTcStages % ksplit ||
      ldh < n_out || size_t(out_tiles) * n_tile < size_t(n_out))
    return cudaErrorInvalidValue;
  ks_round_kernel<<<dim3((n_out + 31) / 32, kRingN / 32), 256, 0, st>>>(acc, outs, mode, n_out, h,
                                                                         ldh);
  cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return le;
  cudaError_t e = cudaFuncSetAttribute(keyswitch_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(TcSmem::kTotal));
  if (e != cudaSuccess) return e;
  const dim3 grid(kTcWordTiles, out_tiles, ksplit);
  keyswitch_tc_kernel<<<grid, kTcThreads, TcSmem::kTotal, st>>>(
      acc, h, ldh, reinterpret_cast<const uint8_t *>(planes), outs, out, n_out, mode, n_tile,
      kTcStages / ksplit, err);
  return cudaGetLastError();
}

}  // namespace ce
