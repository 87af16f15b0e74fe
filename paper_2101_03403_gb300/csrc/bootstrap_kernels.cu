// GPU kernels of the gate-bootstrapping path (sm_103a):
//   lincomb_modswitch  — gate linear combination + modulus switch to 2N
//   blind_rotate       — persistent batched blind rotation (n CMux steps)
//   extract_keyswitch  — fused sample extraction + LWE key switching
//   bsk_to_transform   — bootstrapping key to the transform domain (admission)
//   negacyclic_mul     — exact digit x key products (verification entry point)
// The bootstrapping construction is the TFHE one the paper builds its gates
// on (§3 "TFHE Library": one bootstrap per binary gate, two for MUX).
#include <cuda_runtime.h>

#include <cstdint>

#include "bounded_wait.cuh"
#include "ce_internal.h"
#include "launch.h"
#include "rns_ntt.cuh"

static_assert(ce::kTwistEntries == size_t(rns::kTwEntries), "factor table size");

namespace ce {

namespace {

// Gate linear parts (0, kappa/8) + s1 c1 + s2 c2 (truth tables: §3, Table
// "TFHE API Benchmark"; constants give each row the largest margin from the
// decision boundaries for +-1/8 inputs).  Index 10 = the first MUX half
// (AND of a, b), 11 = the second (ANDNY of a, c).
__constant__ int8_t c_kappa8[12] = {1, -1, 1, 2, -1, -2, -1, -1, 1, 1, -1, -1};
__constant__ int8_t c_s1[12] = {-1, 1, 1, 2, -1, -2, -1, 1, -1, 1, 1, -1};
__constant__ int8_t c_s2[12] = {-1, 1, 1, 2, -1, -2, 1, -1, 1, -1, 1, 1};

// Gadget decomposition offset: rounding to 30 bits (+2^1) plus Bg/2 at each
// of the three digit positions (2^31 + 2^21 + 2^11).  Digit p (1..3) of x is
// ((x + offset) >> (32 - 10 p) & 1023) - 512.
constexpr uint32_t kDecompOffset = 0x80200802u;

// ------------------------------------------------------------------- K1 ---
// One block per job: the gate's linear combination of its two inputs and the
// modulus switch of every word, abar = round(x * 2048 / 2^32) mod 2048.
// mode 0: job g = gate ops[g](a[g], b[g]).  mode 1: MUX, job 2i = AND-part of
// (a[i], b[i]), job 2i+1 = ANDNY-part of (a[i], c[i]).
__global__ void __launch_bounds__(512) lincomb_modswitch_kernel(
    const uint8_t *__restrict__ ops, const uint32_t *__restrict__ a,
    const uint32_t *__restrict__ b, const uint32_t *__restrict__ c,
    uint16_t *__restrict__ abar, int mode, int *__restrict__ err) {
  const int job = blockIdx.x;
  int op, src1, src2;
  const uint32_t *second = b;
  if (mode == 0) {
    op = ops[job];
    if (op > 9) {  // not a gate opcode: flag it and evaluate NAND instead
      if (threadIdx.x == 0) atomicExch(err, 2);
      op = 0;
    }
    src1 = src2 = job;
  } else {
    op = 10 + (job & 1);
    src1 = src2 = job >> 1;
    if (job & 1) second = c;
  }
  const int m = threadIdx.x;
  if (m < kLweWords) {
    const uint32_t x = uint32_t(int32_t(c_s1[op])) * a[size_t(src1) * kLweWords + m] +
                       uint32_t(int32_t(c_s2[op])) * second[size_t(src2) * kLweWords + m] +
                       (m == kLweN ? uint32_t(int32_t(c_kappa8[op])) * kMuEighth : 0u);
    abar[size_t(job) * kAbarStride + m] = uint16_t(((x + (1u << 20)) >> 21) & 2047u);
  }
}

// Gather variant for the netlist engine: job j reads its two inputs from
// arena slots (kSlotWords words each), with optional negation (NOT is free:
// it flips the sign of the input's weight).  op 10/11 are the two halves of
// a MUX (AND-part with (s, x), ANDNY-part with (s, y)).
__global__ void __launch_bounds__(512) lincomb_gather_kernel(const GateJob *__restrict__ jobs,
                                                             const uint32_t *__restrict__ arena,
                                                             uint16_t *__restrict__ abar,
                                                             int *__restrict__ err) {
  const int job = blockIdx.x;
  const GateJob J = jobs[job];
  int op = J.op;
  if (op > 11) {
    if (threadIdx.x == 0) atomicExch(err, 2);
    op = 0;
  }
  const int m = threadIdx.x;
  if (m < kLweWords) {
    const uint32_t w1 = uint32_t(int32_t(c_s1[op]) * (J.neg_a ? -1 : 1));
    const uint32_t w2 = uint32_t(int32_t(c_s2[op]) * (J.neg_b ? -1 : 1));
    const uint32_t x = w1 * arena[size_t(J.a) * kSlotWords + m] +
                       w2 * arena[size_t(J.b) * kSlotWords + m] +
                       (m == kLweN ? uint32_t(int32_t(c_kappa8[op])) * kMuEighth : 0u);
    abar[size_t(job) * kAbarStride + m] = uint16_t(((x + (1u << 20)) >> 21) & 2047u);
  }
}

// ------------------------------------------------------------------- K2 ---
// Persistent batched blind rotation.  A block holds G gates (128 threads
// each) and streams the bootstrapping key once per block: the transform-
// domain rows of CMux step i, gadget level p (4 polynomials, 32 KB) arrive by
// bulk asynchronous copy into a ring of NSLOT shared-memory slots and are
// used by all G gates.  The last warp to finish with a slot refills it.
// Each gate's group synchronises only itself (named barrier 1 + g), so the
// groups drift within the ring's slack and their multiply-heavy and
// add-heavy phases overlap on the SM's two integer pipes.
//
// Per gate and step i (a CMux controlled by key bit s_i): D = X^abar_i ACC -
// ACC; for p = 1..3: forward-transform digit p of both halves of D, multiply
// by the key rows and accumulate in the transform domain; then one inverse
// transform of the two accumulators and ACC += result (exact mod 2^32).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait for a slot's copy (bounded_wait.cuh); on expiry the block
// records the error, raises its abort flag and continues without waiting
// (results are then invalid and the host reports CE_ETIMEOUT).
__device__ __forceinline__ void wait_slot(uint32_t bar, uint32_t parity, volatile int *abort,
                                          int *err) {
  (void)bounded_wait(bar, parity, abort, err);
}

__device__ __forceinline__ void issue_chunk(uint64_t *slot, uint32_t bar, const uint64_t *src) {
  constexpr uint32_t kBytes = kChunkWords * 8;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(slot)),
      "l"(src), "r"(kBytes), "r"(bar)
      : "memory");
}

template <int G, int NSLOT>
struct BrSmem {
  static constexpr size_t kRing = size_t(NSLOT) * kChunkWords * 8;
  static constexpr size_t kAcc = 2 * kRingN * 4;                 // per gate
  static constexpr size_t kBuf = size_t(rns::kBufWords) * 8;     // per gate
  static constexpr size_t kGate = kAcc + kBuf;
  static constexpr size_t kBars = 64;
  static constexpr size_t kTotal = kRing + G * kGate + kBars + 64;
};

template <int G, int NSLOT>
__global__ void __launch_bounds__(128 * G, 1) blind_rotate_kernel(
    const uint64_t *__restrict__ bsk, const uint64_t *const *__restrict__ grp_bsk,
    const uint16_t *__restrict__ abar, uint32_t *__restrict__ acc_out, int n_jobs,
    const uint4 *__restrict__ tw, int *__restrict__ err, int key_base, int key_div) {
  using L = BrSmem<G, NSLOT>;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *ring = reinterpret_cast<uint64_t *>(smem);
  const int g = threadIdx.x >> 7, t = threadIdx.x & 127, lane = threadIdx.x & 31;
  uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L::kRing + g * L::kGate);
  uint2 *buf = reinterpret_cast<uint2 *>(smem + L::kRing + g * L::kGate + L::kAcc);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::kRing + G * L::kGate);
  uint32_t *count = reinterpret_cast<uint32_t *>(full + NSLOT);
  volatile int *abort = reinterpret_cast<volatile int *>(count + NSLOT);
  constexpr int kChunksPerGate = kLweN * kGadgetL;  // 1500
  constexpr int kWarps = 4 * G;

  const int n_groups = (n_jobs + G - 1) / G;
  const int my_groups =
      blockIdx.x < n_groups ? (n_groups - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int total_chunks = my_groups * kChunksPerGate;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSLOT; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + s)) : "memory");
      count[s] = 0;
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // Key of the gate group that consumes chunk c of this block (all gates of
  // a group belong to the same client): grp_bsk[(key_base + first job of
  // the group) / key_div], key_base = this launch's first job in the batch.
  auto chunk_src = [&](int c) {
    const uint64_t *key = bsk;
    if (grp_bsk)
      key = grp_bsk[(key_base + (int(blockIdx.x) + (c / kChunksPerGate) * int(gridDim.x)) * G) /
                    key_div];
    return key + size_t(c % kChunksPerGate) * kChunkWords;
  };
  if (threadIdx.x == 0) {
    for (int c = 0; c < NSLOT && c < total_chunks; ++c)
      issue_chunk(ring + size_t(c) * kChunkWords, smem_u32(full + c), chunk_src(c));
  }

  const int P = t >> 6, n1 = t & 63;
  int chunk = 0;
  for (int jg = 0; jg < my_groups; ++jg) {
    const int job = (blockIdx.x + jg * gridDim.x) * G + g;
    const bool active = job < n_jobs;
    const uint16_t *ab = abar + size_t(active ? job : 0) * kAbarStride;

    // ACC = (0, X^(-bbar) v), v = mu * sum_j X^j, mu = +1/8.
    {
      const int bbar = active ? ab[kLweN] : 0;
      const int k = (2 * kRingN - bbar) & (2 * kRingN - 1);
      for (int j = t; j < kRingN; j += 128) {
        acc[j] = 0;
        const bool hi = k < kRingN ? (j >= k) : (j < k - kRingN);
        acc[kRingN + j] = hi ? kMuEighth : 0u - kMuEighth;
      }
    }
    rns::named_bar(1 + g, 128);

    for (int i = 0; i < kLweN; ++i) {
      // A zero rotation (or an inactive slot) gives D = 0, whose digits are
      // all zero, so the step adds exactly zero.
      const int rot = active ? __ldg(ab + i) : 0;
      uint32_t w[16];
      uint64_t XL[2][2][8];  // [prime][output polynomial][position], unreduced key sums
      {
        // w = X^rot ACC_P - ACC_P + decomposition offset, at n = n1 + 64 n2.
        const uint32_t *src = acc + P * kRingN;
        const int kk = rot & (kRingN - 1);
        const uint32_t flip = (rot >= kRingN) ? 0xFFFFFFFFu : 0u;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
          const int n = n1 + 64 * n2;
          const int s = n - kk;
          uint32_t r = s >= 0 ? src[s] : 0u - src[s + kRingN];
          r = (r ^ flip) - flip;  // negate when rot >= N (X^N = -1)
          w[n2] = r - src[n] + kDecompOffset;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int o = 0; o < 2; ++o)
#pragma unroll
            for (int d = 0; d < 8; ++d) XL[q][o][d] = 0;
      }
#pragma unroll 1
      for (int pz = 0; pz < kGadgetL; ++pz, ++chunk) {
        const int slot = chunk % NSLOT;
        uint32_t v[2][16], Y[2][2][8];
        const int sh = 22 - 10 * pz;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
          // digit + 512 in [0, 1024); digit + p lies in (0, 2p).
          const uint32_t u = (w[n2] >> sh) & 1023u;
          v[0][n2] = rns::pretwist<0>(u + (rns::P<0>() - 512u), n2);
          v[1][n2] = rns::pretwist<1>(u + (rns::P<1>() - 512u), n2);
        }
        rns::forward(v, Y, buf, t, 1 + g, 128, tw);
        wait_slot(smem_u32(full + slot), uint32_t(chunk / NSLOT) & 1u, abort, err);
        // X[o] += Y[0] * key(c=0, p, o) + Y[1] * key(c=1, p, o), per prime;
        // key words are (k mod p0, k mod p1) in Montgomery form, positions d
        // and d+1 in one 16-byte word.
        const uint4 *key = reinterpret_cast<const uint4 *>(ring + size_t(slot) * kChunkWords) + t;
#pragma unroll
        for (int dp = 0; dp < 4; ++dp) {
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            const uint4 k0 = key[((0 * 2 + o) * 4 + dp) * 128];
            const uint4 k1 = key[((1 * 2 + o) * 4 + dp) * 128];
            const int d = 2 * dp;
            XL[0][o][d] += uint64_t(Y[0][0][d]) * k0.x + uint64_t(Y[0][1][d]) * k1.x;
            XL[1][o][d] += uint64_t(Y[1][0][d]) * k0.y + uint64_t(Y[1][1][d]) * k1.y;
            XL[0][o][d + 1] += uint64_t(Y[0][0][d + 1]) * k0.z + uint64_t(Y[0][1][d + 1]) * k1.z;
            XL[1][o][d + 1] += uint64_t(Y[1][0][d + 1]) * k0.w + uint64_t(Y[1][1][d + 1]) * k1.w;
          }
        }
        // Release the slot; the last warp out refills it with chunk + NSLOT.
        __syncwarp();
        if (lane == 0) {
          __threadfence_block();
          const uint32_t old = atomicAdd(count + slot, 1u);
          if (old == kWarps - 1) {
            count[slot] = 0;
            __threadfence_block();
            const int next = chunk + NSLOT;
            if (next < total_chunks && !*abort)
              issue_chunk(ring + size_t(slot) * kChunkWords, smem_u32(full + slot),
                          chunk_src(next));
          }
        }
      }
      {
        // six products of a value below 16p and a key below p: below 96 p^2
        // < 2^63; one Montgomery reduction gives below 96 p^2 / 2^32 + p < 7p,
        // which the inverse takes
        uint32_t X[2][2][8], v[2][16];
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            X[0][o][d] = rns::redc<0>(XL[0][o][d]);
            X[1][o][d] = rns::redc<1>(XL[1][o][d]);
          }
        rns::inverse(X, v, buf, t, 1 + g, 128, tw);
        uint32_t *dst = acc + P * kRingN + n1;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) dst[64 * n2] += rns::lift32(v[0][n2], v[1][n2]);
      }
      rns::named_bar(1 + g, 128);
    }
    if (active) {
      uint32_t *out = acc_out + size_t(job) * 2 * kRingN;
      for (int j = t; j < 2 * kRingN; j += 128) out[j] = acc[j];
    }
    rns::named_bar(1 + g, 128);
  }
}

// Latency-oriented blind rotation: one gate per block, three 128-thread
// groups.  In each CMux step group g forward-transforms gadget level g of
// both accumulator halves and multiplies by its key chunk (kept in its own
// shared-memory slot, refilled by bulk copy for the next step right after
// use); groups 1 and 2 hand their partial sums to group 0 through shared
// memory, and group 0 runs the inverse transform and updates ACC.  The step's
// critical path is one forward transform, one exchange and one inverse
// instead of three forward transforms and one inverse.
struct WideSmem {
  static constexpr size_t kSlots = size_t(3) * kChunkWords * 8;
  static constexpr size_t kAcc = 2 * kRingN * 4;
  static constexpr size_t kBufs = size_t(3) * rns::kBufWords * 8;
  static constexpr size_t kXch = size_t(2) * 2 * 8 * 128 * 8;
  static constexpr size_t kTotal = kSlots + kAcc + kBufs + kXch + 64;
};

__global__ void __launch_bounds__(384, 1) blind_rotate_wide_kernel(
    const uint64_t *__restrict__ bsk, const uint64_t *const *__restrict__ gate_bsk,
    const uint16_t *__restrict__ abar, uint32_t *__restrict__ acc_out, int n_jobs,
    const uint4 *__restrict__ tw, int *__restrict__ err, int key_base, int key_div) {
  using L = WideSmem;
  extern __shared__ __align__(128) uint8_t smem[];
  uint64_t *slots = reinterpret_cast<uint64_t *>(smem);
  uint32_t *acc = reinterpret_cast<uint32_t *>(smem + L::kSlots);
  uint2 *bufs = reinterpret_cast<uint2 *>(smem + L::kSlots + L::kAcc);
  uint2 *xch = reinterpret_cast<uint2 *>(smem + L::kSlots + L::kAcc + L::kBufs);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::kSlots + L::kAcc + L::kBufs + L::kXch);
  volatile int *abort = reinterpret_cast<volatile int *>(full + 3);
  const int g = threadIdx.x >> 7, t = threadIdx.x & 127;
  uint2 *buf = bufs + g * rns::kBufWords;
  uint64_t *slot = slots + size_t(g) * kChunkWords;
  const int my_gates = int(blockIdx.x) < n_jobs ? (n_jobs - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const int total = my_gates * kLweN;  // chunks per group
  auto chunk_src = [&](int c) {
    const int gate = blockIdx.x + (c / kLweN) * gridDim.x;
    const uint64_t *key = gate_bsk ? gate_bsk[(key_base + gate) / key_div] : bsk;
    return key + (size_t(c % kLweN) * kGadgetL + g) * kChunkWords;
  };
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(full + k)) : "memory");
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0 && total > 0) issue_chunk(slot, smem_u32(full + g), chunk_src(0));
  const int P = t >> 6, n1 = t & 63;
  int c = 0;
  for (int jg = 0; jg < my_gates; ++jg) {
    const int job = blockIdx.x + jg * gridDim.x;
    const uint16_t *ab = abar + size_t(job) * kAbarStride;
    {
      const int bbar = ab[kLweN];
      const int k = (2 * kRingN - bbar) & (2 * kRingN - 1);
      for (int j = threadIdx.x; j < kRingN; j += 384) {
        acc[j] = 0;
        const bool hi = k < kRingN ? (j >= k) : (j < k - kRingN);
        acc[kRingN + j] = hi ? kMuEighth : 0u - kMuEighth;
      }
    }
    __syncthreads();
    for (int i = 0; i < kLweN; ++i, ++c) {
      const int rot = __ldg(ab + i);
      uint32_t v[2][16], Y[2][2][8];
      {
        const uint32_t *src = acc + P * kRingN;
        const int kk = rot & (kRingN - 1);
        const uint32_t flip = (rot >= kRingN) ? 0xFFFFFFFFu : 0u;
        const int sh = 22 - 10 * g;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) {
          const int n = n1 + 64 * n2;
          const int sidx = n - kk;
          uint32_t r = sidx >= 0 ? src[sidx] : 0u - src[sidx + kRingN];
          r = (r ^ flip) - flip;
          const uint32_t wv = r - src[n] + kDecompOffset;
          const uint32_t u = (wv >> sh) & 1023u;  // digit + 512
          v[0][n2] = rns::pretwist<0>(u + (rns::P<0>() - 512u), n2);
          v[1][n2] = rns::pretwist<1>(u + (rns::P<1>() - 512u), n2);
        }
      }
      rns::forward(v, Y, buf, t, 1 + g, 128, tw);
      wait_slot(smem_u32(full + g), uint32_t(c) & 1u, abort, err);
      uint32_t X[2][2][8];  // this level's products, each below 3p
      {
        const uint4 *key = reinterpret_cast<const uint4 *>(slot) + t;
#pragma unroll
        for (int dp = 0; dp < 4; ++dp)
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            const uint4 k0 = key[((0 * 2 + o) * 4 + dp) * 128];
            const uint4 k1 = key[((1 * 2 + o) * 4 + dp) * 128];
            const int d = 2 * dp;
            X[0][o][d] = rns::redc<0>(uint64_t(Y[0][0][d]) * k0.x + uint64_t(Y[0][1][d]) * k1.x);
            X[1][o][d] = rns::redc<1>(uint64_t(Y[1][0][d]) * k0.y + uint64_t(Y[1][1][d]) * k1.y);
            X[0][o][d + 1] =
                rns::redc<0>(uint64_t(Y[0][0][d + 1]) * k0.z + uint64_t(Y[0][1][d + 1]) * k1.z);
            X[1][o][d + 1] =
                rns::redc<1>(uint64_t(Y[1][0][d + 1]) * k0.w + uint64_t(Y[1][1][d + 1]) * k1.w);
          }
      }
      rns::named_bar(1 + g, 128);  // the group is done with its slot
      if (t == 0 && c + 1 < total && !*abort) issue_chunk(slot, smem_u32(full + g), chunk_src(c + 1));
      if (g > 0) {
        uint2 *x = xch + size_t(g - 1) * 2 * 8 * 128 + t;
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int d = 0; d < 8; ++d) x[(o * 8 + d) * 128] = make_uint2(X[0][o][d], X[1][o][d]);
      }
      __syncthreads();
      if (g == 0) {
        const uint2 *x1 = xch + t, *x2 = xch + 2 * 8 * 128 + t;
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int d = 0; d < 8; ++d) {
            // three terms below 3p: below 9p, which the inverse takes
            const uint2 a1 = x1[(o * 8 + d) * 128], a2 = x2[(o * 8 + d) * 128];
            X[0][o][d] = X[0][o][d] + a1.x + a2.x;
            X[1][o][d] = X[1][o][d] + a1.y + a2.y;
          }
        rns::inverse(X, v, buf, t, 1, 128, tw);
        uint32_t *dst = acc + P * kRingN + n1;
#pragma unroll
        for (int n2 = 0; n2 < 16; ++n2) dst[64 * n2] += rns::lift32(v[0][n2], v[1][n2]);
      }
      __syncthreads();
    }
    uint32_t *out = acc_out + size_t(job) * 2 * kRingN;
    for (int j = threadIdx.x; j < 2 * kRingN; j += 384) out[j] = acc[j];
    __syncthreads();
  }
}

// ------------------------------------------------------------------- K4 ---
// Fused sample extraction (coefficient 0: a'_0 = A_0, a'_j = -A_{N-j},
// b' = B_0) and key switching: each a'_j rounded to 16 bits, split into 8
// base-4 digits (most significant first), out = (0, b') - sum KSK[j][q][digit].
// A block serves GT outputs for a range of j; the three KSK rows of (j, q) are
// read once (uint4 per thread) and applied to all GT outputs.  With several
// j-ranges the partial sums are added atomically (exact mod 2^32; the
// outputs start at zero).  An output combines one accumulator, or two plus
// (0, +1/8) for a MUX, before switching.  MODE 0: output o = job o, packed
// [n][501] output; MODE 1: MUX, jobs 2o and 2o+1, packed output; MODE 2:
// descriptors (jobs, arena slot) from `outs`, written to the arena.  With
// tile_ksk set, tile t uses the key tile_ksk[t] (one client per tile).
template <int GT, int MODE>
__global__ void __launch_bounds__(128) extract_keyswitch_kernel(
    const uint32_t *__restrict__ acc, const uint32_t *__restrict__ ksk_one,
    const uint32_t *const *__restrict__ tile_ksk, const GateOut *__restrict__ outs,
    uint32_t *__restrict__ out, int n_out, int jchunk) {
  extern __shared__ uint16_t hbits[];  // [GT][jchunk]
  const int tile = blockIdx.x, j0 = blockIdx.y * jchunk;
  const int j1 = min(kRingN, j0 + jchunk);
  const uint32_t *ksk = tile_ksk ? tile_ksk[tile] : ksk_one;
  auto jobs_of = [&](int o, int &j1x, int &j2x) {
    if (MODE == 0) { j1x = o; j2x = -1; }
    else if (MODE == 1) { j1x = 2 * o; j2x = 2 * o + 1; }
    else { j1x = outs[o].job1; j2x = outs[o].job2; }
  };
  for (int idx = threadIdx.x; idx < GT * jchunk; idx += 128) {
    const int g = idx / jchunk, j = j0 + idx % jchunk;
    const int o = tile * GT + g;
    uint32_t h = 0;
    if (o < n_out && j < j1) {
      int ja, jb;
      jobs_of(o, ja, jb);
      const uint32_t *A = acc + size_t(ja) * 2 * kRingN;
      uint32_t aj = (j == 0) ? A[0] : 0u - A[kRingN - j];
      if (jb >= 0) {
        const uint32_t *A2 = acc + size_t(jb) * 2 * kRingN;
        aj += (j == 0) ? A2[0] : 0u - A2[kRingN - j];
      }
      h = (aj + 0x8000u) >> 16;
    }
    hbits[idx] = uint16_t(h);
  }
  __syncthreads();

  uint32_t s[GT][4];
#pragma unroll
  for (int g = 0; g < GT; ++g)
#pragma unroll
    for (int e = 0; e < 4; ++e) s[g][e] = 0;
  const uint4 *K = reinterpret_cast<const uint4 *>(ksk) + threadIdx.x;
#pragma unroll 1
  for (int j = j0; j < j1; ++j) {
#pragma unroll 2
    for (int q = 0; q < kKsT; ++q) {
      const size_t row = (size_t(j) * kKsT + q) * 3;
      const uint4 k1 = __ldg(K + (row + 0) * (kKskRow / 4));
      const uint4 k2 = __ldg(K + (row + 1) * (kKskRow / 4));
      const uint4 k3 = __ldg(K + (row + 2) * (kKskRow / 4));
      const int shift = 14 - 2 * q;
#pragma unroll
      for (int g = 0; g < GT; ++g) {
        const uint32_t dg = (uint32_t(hbits[g * jchunk + (j - j0)]) >> shift) & 3u;
        const uint4 sel = dg == 1 ? k1 : (dg == 2 ? k2 : k3);
        const uint32_t m = dg ? 0xFFFFFFFFu : 0u;
        s[g][0] += sel.x & m;
        s[g][1] += sel.y & m;
        s[g][2] += sel.z & m;
        s[g][3] += sel.w & m;
      }
    }
  }
#pragma unroll
  for (int g = 0; g < GT; ++g) {
    const int o = tile * GT + g;
    if (o >= n_out) break;
    int ja, jb;
    jobs_of(o, ja, jb);
    uint32_t *dst = MODE == 2 ? out + size_t(outs[o].slot) * kSlotWords : out + size_t(o) * kLweWords;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int m = 4 * threadIdx.x + e;
      if (m >= kLweWords) continue;
      uint32_t val = 0u - s[g][e];
      if (m == kLweN && blockIdx.y == 0) {
        uint32_t bp = acc[size_t(ja) * 2 * kRingN + kRingN];
        if (jb >= 0) bp += acc[size_t(jb) * 2 * kRingN + kRingN] + kMuEighth;
        val += bp;
      }
      if (gridDim.y == 1)
        dst[m] = val;
      else
        atomicAdd(dst + m, val);
    }
  }
}

// Zeroes the output words of descriptor-addressed outputs (before a split
// key switch accumulates into them atomically).
__global__ void zero_slots_kernel(const GateOut *__restrict__ outs, uint32_t *__restrict__ arena) {
  const uint32_t slot = outs[blockIdx.x].slot;
  for (int m = threadIdx.x; m < kLweWords; m += blockDim.x) arena[size_t(slot) * kSlotWords + m] = 0;
}

// --------------------------------------------------------- key to transform ---
// Block (i, p): transforms the four polynomials (TRGSW half c, component o)
// of bootstrapping-key rows r = c*3 + p of key bit i (coefficients lifted to
// [-2^31, 2^31)) and stores them, reduced and in Montgomery form, in the
// [i][p][c*2+o][d/2][thread][d%2] order the blind rotation reads (one
// 16-byte load gives a thread its positions d and d+1): one 64-bit word per
// position holding the residues (mod p0, mod p1).
__global__ void __launch_bounds__(128) bsk_to_transform_kernel(const uint32_t *__restrict__ bsk,
                                                               uint2 *__restrict__ out,
                                                               const uint4 *__restrict__ tw) {
  __shared__ uint2 buf[rns::kBufWords];
  const int i = blockIdx.x / kGadgetL, pz = blockIdx.x % kGadgetL, t = threadIdx.x;
  const int P = t >> 6, n1 = t & 63;
  for (int c = 0; c < 2; ++c) {
    const uint32_t *row = bsk + ((size_t(i) * 2 * kGadgetL + c * kGadgetL + pz) * 2 + P) * kRingN;
    uint32_t v[2][16], X[2][2][8];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      const int32_t k = int32_t(row[n1 + 64 * n2]);
      v[0][n2] = rns::pretwist<0>(rns::from_i32<0>(k), n2);
      v[1][n2] = rns::pretwist<1>(rns::from_i32<1>(k), n2);
    }
    rns::forward(v, X, buf, t, 1, 128, tw);
    uint2 *dst = out + size_t(blockIdx.x) * kChunkWords;
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int d = 0; d < 8; ++d)
        dst[((c * 2 + o) * 4 + d / 2) * 256 + 2 * t + (d & 1)] =
            make_uint2(rns::fold<0, 1>(rns::to_mont<0>(X[0][o][d])),
                       rns::fold<1, 1>(rns::to_mont<1>(X[1][o][d])));
  }
}

// ---------------------------------------------------------- negacyclic mul ---
// Block b: products 2b and 2b+1 (d signed 16-bit, k uint32), exact mod 2^32.
__global__ void __launch_bounds__(128) negacyclic_mul_kernel(const int16_t *__restrict__ dg,
                                                             const uint32_t *__restrict__ k,
                                                             uint32_t *__restrict__ out, int n,
                                                             const uint4 *__restrict__ tw) {
  __shared__ uint2 buf[rns::kBufWords];
  const int t = threadIdx.x, P = t >> 6, n1 = t & 63;
  const int prod = 2 * blockIdx.x + P;
  const bool live = prod < n;
  uint32_t v[2][16], XD[2][2][8], XK[2][2][8];
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    const int32_t x = live ? dg[size_t(prod) * kRingN + n1 + 64 * n2] : 0;
    v[0][n2] = rns::pretwist<0>(rns::from_i32<0>(x), n2);
    v[1][n2] = rns::pretwist<1>(rns::from_i32<1>(x), n2);
  }
  rns::forward(v, XD, buf, t, 1, 128, tw);
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    const int32_t x = live ? int32_t(k[size_t(prod) * kRingN + n1 + 64 * n2]) : 0;
    v[0][n2] = rns::pretwist<0>(rns::from_i32<0>(x), n2);
    v[1][n2] = rns::pretwist<1>(rns::from_i32<1>(x), n2);
  }
  rns::forward(v, XK, buf, t, 1, 128, tw);
  // XD * XK = redc(XD * mont(XK)): XD < 16p and mont(XK) < 2p keep the
  // product below 32 p^2 < 2^61 and the reduction below 3p.
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      XD[0][q][d] = rns::redc<0>(uint64_t(XD[0][q][d]) * rns::to_mont<0>(XK[0][q][d]));
      XD[1][q][d] = rns::redc<1>(uint64_t(XD[1][q][d]) * rns::to_mont<1>(XK[1][q][d]));
    }
  rns::inverse(XD, v, buf, t, 1, 128, tw);
  if (live) {
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2)
      out[size_t(prod) * kRingN + n1 + 64 * n2] = rns::lift32(v[0][n2], v[1][n2]);
  }
}

template <int G, int NSLOT>
cudaError_t launch_br(const uint64_t *bsk, const uint64_t *const *grp_bsk, const uint16_t *abar,
                      uint32_t *acc, int n, const uint4 *tw, int *err, int blocks,
                      cudaStream_t st, int key_base, int key_div) {
  using L = BrSmem<G, NSLOT>;
  auto kern = blind_rotate_kernel<G, NSLOT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(L::kTotal));
  if (e != cudaSuccess) return e;
  kern<<<blocks, 128 * G, L::kTotal, st>>>(bsk, grp_bsk, abar, acc, n, tw, err, key_base,
                                           key_div);
  return cudaGetLastError();
}

// One launch of shape G over jobs [key_base, key_base + n) of the batch
// (abar and acc already offset to the first of them).
cudaError_t launch_shape(int G, const uint64_t *bsk, const uint64_t *const *grp_bsk,
                         const uint16_t *abar, uint32_t *acc, int n, const uint4 *tw, int *err,
                         int blocks, cudaStream_t st, int key_base, int key_div) {
  switch (G) {
    case 1: return launch_br<1, 2>(bsk, grp_bsk, abar, acc, n, tw, err, blocks, st, key_base, key_div);
    case 2: return launch_br<2, 3>(bsk, grp_bsk, abar, acc, n, tw, err, blocks, st, key_base, key_div);
    case 3: {  // one gate per block, three cooperating groups
      cudaError_t e = cudaFuncSetAttribute(blind_rotate_wide_kernel,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           int(WideSmem::kTotal));
      if (e != cudaSuccess) return e;
      blind_rotate_wide_kernel<<<blocks, 384, WideSmem::kTotal, st>>>(bsk, grp_bsk, abar, acc, n,
                                                                      tw, err, key_base, key_div);
      return cudaGetLastError();
    }
    default: return launch_br<4, 3>(bsk, grp_bsk, abar, acc, n, tw, err, blocks, st, key_base, key_div);
  }
}

}  // namespace

size_t blind_rotate_smem_bytes(int gates_per_block) {
  switch (gates_per_block) {
    case 1: return BrSmem<1, 2>::kTotal;
    case 2: return BrSmem<2, 3>::kTotal;
    case 3: return WideSmem::kTotal;
    default: return BrSmem<4, 3>::kTotal;
  }
}

cudaError_t launch_lincomb_modswitch(const uint8_t *ops, const uint32_t *a, const uint32_t *b,
                                     const uint32_t *c, uint16_t *abar, int n_jobs, int mode,
                                     int *err, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  lincomb_modswitch_kernel<<<n_jobs, 512, 0, st>>>(ops, a, b, c, abar, mode, err);
  return cudaGetLastError();
}

BrSplit blind_rotate_split(int n_jobs, int G, int blocks) {
  BrSplit s{n_jobs, 0, 0, 0};
  const int gsz = G == 3 ? 1 : G;
  const int groups = (n_jobs + gsz - 1) / gsz;
  if ((G != 4 && G != 2) || blocks <= 0 || groups <= blocks || groups % blocks == 0) return s;
  const int main_jobs = (groups / blocks) * blocks * gsz;  // the whole rounds
  const int tail = n_jobs - main_jobs;
  if (tail <= blocks) {  // one gate per block (latency shape): ~0.4 (G 4) / ~0.6 (G 2) of a round
    s = BrSplit{main_jobs, tail, 3, tail};
  } else if (G == 4 && tail <= 2 * blocks) {  // two gates per block: ~0.6 of a round
    s = BrSplit{main_jobs, tail, 2, (tail + 1) / 2};
  }
  return s;
}

cudaError_t launch_blind_rotate(const uint64_t *bsk, const uint16_t *abar, uint32_t *acc,
                                int n_jobs, const uint4 *tw, int *err, int gates_per_block,
                                int blocks, cudaStream_t st, const uint64_t *const *grp_bsk,
                                int *launches) {
  if (n_jobs <= 0) return cudaSuccess;
  const int gsz = gates_per_block == 3 ? 1 : gates_per_block;
  const BrSplit s = blind_rotate_split(n_jobs, gates_per_block, blocks);
  cudaError_t e = launch_shape(gates_per_block, bsk, grp_bsk, abar, acc, s.main_jobs, tw, err,
                               blocks, st, 0, gsz);
  if (launches) ++*launches;
  if (e != cudaSuccess || s.tail_jobs == 0) return e;
  e = launch_shape(s.tail_G, bsk, grp_bsk, abar + size_t(s.main_jobs) * kAbarStride,
                   acc + size_t(s.main_jobs) * 2 * kRingN, s.tail_jobs, tw, err, s.tail_blocks,
                   st, s.main_jobs, gsz);
  if (launches) ++*launches;
  return e;
}

template <int GT>
void launch_ks_tile(int mode, dim3 grid, size_t sm, cudaStream_t st, const uint32_t *acc,
                    const uint32_t *ksk, const uint32_t *const *tile_ksk, const GateOut *outs,
                    uint32_t *out, int n_out, int jchunk) {
  if (mode == 0)
    extract_keyswitch_kernel<GT, 0><<<grid, 128, sm, st>>>(acc, ksk, tile_ksk, outs, out, n_out, jchunk);
  else if (mode == 1)
    extract_keyswitch_kernel<GT, 1><<<grid, 128, sm, st>>>(acc, ksk, tile_ksk, outs, out, n_out, jchunk);
  else
    extract_keyswitch_kernel<GT, 2><<<grid, 128, sm, st>>>(acc, ksk, tile_ksk, outs, out, n_out, jchunk);
}

cudaError_t launch_extract_keyswitch(const uint32_t *acc, const uint32_t *ksk, uint32_t *out,
                                     int n_out, bool mux, int tile, int jsplit, cudaStream_t st) {
  return launch_extract_keyswitch_ex(acc, ksk, nullptr, nullptr, out, n_out, mux ? 1 : 0, tile,
                                     jsplit, st);
}

cudaError_t launch_extract_keyswitch_ex(const uint32_t *acc, const uint32_t *ksk,
                                        const uint32_t *const *tile_ksk, const GateOut *outs,
                                        uint32_t *out, int n_out, int mode, int tile, int jsplit,
                                        cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  const int jchunk = (kRingN + jsplit - 1) / jsplit;
  const dim3 grid((n_out + tile - 1) / tile, jsplit);
  const size_t sm = size_t(tile) * jchunk * sizeof(uint16_t);
  if (tile == 1) launch_ks_tile<1>(mode, grid, sm, st, acc, ksk, tile_ksk, outs, out, n_out, jchunk);
  else if (tile == 4) launch_ks_tile<4>(mode, grid, sm, st, acc, ksk, tile_ksk, outs, out, n_out, jchunk);
  else launch_ks_tile<16>(mode, grid, sm, st, acc, ksk, tile_ksk, outs, out, n_out, jchunk);
  return cudaGetLastError();
}

cudaError_t launch_lincomb_gather(const GateJob *jobs, const uint32_t *arena, uint16_t *abar,
                                  int n_jobs, int *err, cudaStream_t st) {
  if (n_jobs <= 0) return cudaSuccess;
  lincomb_gather_kernel<<<n_jobs, 512, 0, st>>>(jobs, arena, abar, err);
  return cudaGetLastError();
}

cudaError_t launch_zero_slots(const GateOut *outs, uint32_t *arena, int n_out, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  zero_slots_kernel<<<n_out, 128, 0, st>>>(outs, arena);
  return cudaGetLastError();
}

cudaError_t launch_bsk_to_transform(const uint32_t *bsk, uint64_t *out, const uint4 *tw,
                                    cudaStream_t st) {
  bsk_to_transform_kernel<<<kLweN * kGadgetL, 128, 0, st>>>(bsk, reinterpret_cast<uint2 *>(out),
                                                             tw);
  return cudaGetLastError();
}

// Failure-detection self-test: one thread waits on an mbarrier whose phase
// nothing completes (one expected arrival, none made), with the library's
// bounded wait and a short limit; the wait expires and raises the error flag.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int *err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    abort_flag = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) (void)bounded_wait(smem_addr(&bar), 0u, &abort_flag, err, limit_ns);
}

// Integer multiply-add pipe probe: every thread runs eight independent chains
// of `iters` dependent operations of one kind on per-thread operands (0:
// 32-bit multiply-add, 1:
// high half of a 32 x 32-bit product plus an addend, 2: 32 x 32 -> 64-bit
// product plus a 64-bit addend) between two reads of the SM clock; block b
// stores its cycle count and the SM it ran on.  Launched with every block
// resident at once.
template <int KIND>
__global__ void __launch_bounds__(512) int_pipe_probe_kernel(uint32_t a, uint32_t b, int iters,
                                                             uint32_t *sink, long long *cycles,
                                                             int *smid) {
  // per-thread operands (registers, as the transform's factors are)
  a ^= threadIdx.x << 1;
  b += threadIdx.x;
  uint32_t x[8];
  uint64_t y[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = threadIdx.x * 2654435761u + uint32_t(k) * 7919u;
    y[k] = x[k];
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (KIND == 0) x[k] = x[k] * a + b;
      if (KIND == 1) x[k] = __umulhi(x[k], a) + b;
      if (KIND == 2) y[k] = uint64_t(uint32_t(y[k])) * a + y[k];
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t f = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) f ^= x[k] ^ uint32_t(y[k]) ^ uint32_t(y[k] >> 32);
  sink[size_t(blockIdx.x) * blockDim.x + threadIdx.x] = f;
  if (threadIdx.x == 0) {
    cycles[blockIdx.x] = t1 - t0;
    int id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    smid[blockIdx.x] = id;
  }
}

cudaError_t launch_int_pipe_probe(int kind, int blocks, int threads, int iters, uint32_t *sink,
                                  long long *cycles, int *smid, cudaStream_t st) {
  const uint32_t a = 0x9E3779B1u, b = 0x7F4A7C15u;
  if (kind == 0)
    int_pipe_probe_kernel<0><<<blocks, threads, 0, st>>>(a, b, iters, sink, cycles, smid);
  else if (kind == 1)
    int_pipe_probe_kernel<1><<<blocks, threads, 0, st>>>(a, b, iters, sink, cycles, smid);
  else
    int_pipe_probe_kernel<2><<<blocks, threads, 0, st>>>(a, b, iters, sink, cycles, smid);
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, int *err, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, err);
  return cudaGetLastError();
}

cudaError_t launch_negacyclic_mul(const int16_t *d, const uint32_t *k, uint32_t *out, int n,
                                  const uint4 *tw, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  negacyclic_mul_kernel<<<(n + 1) / 2, 128, 0, st>>>(d, k, out, n, tw);
  return cudaGetLastError();
}

}  // namespace ce
