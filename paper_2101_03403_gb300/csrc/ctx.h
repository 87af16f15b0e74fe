// The context object behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ce_internal.h"

namespace ce {

constexpr uint64_t kBskNttBytes = kBskNttWords * 8;
constexpr uint64_t kKskDevBytes = kKskDevWords * 4;
// fp16 limb planes of the key-switching key for the tensor-core key switch:
// [4 word tiles][512 stages][3 limbs][128 words x 48] (keyswitch_tc.cu).
constexpr uint64_t kKsPlaneBytes = uint64_t(4) * 512 * 3 * 128 * 48 * 2;
// Coefficient-domain bootstrapping key, kept for the tensor-core external
// product, whose Hankel limb sequences are built from it on first use.
constexpr uint64_t kBskCoefBytes = uint64_t(CE_BSK_WORDS) * 4;
constexpr uint64_t kClientBytes = kBskNttBytes + kKskDevBytes + kKsPlaneBytes + kBskCoefBytes;

struct Client {
  bool live = false;
  uint64_t *bsk = nullptr;  // transform-domain bootstrapping key
  uint32_t *ksk = nullptr;  // [j][q][v-1][512]
  uint16_t *ksk_planes = nullptr;  // fp16 limb planes for the tensor-core key switch
  uint32_t *bsk_coef = nullptr;    // [i][r][o][N] coefficient key
  uint16_t *bsk_hankel = nullptr;  // Hankel limb sequences (tensor-core external product)
};

class Engine;  // netlist engine (engine.cu), created on first use

}  // namespace ce

struct ce_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sms = 0;
  uint64_t budget = 0, used = 0;
  std::vector<ce::Client> clients;
  uint4 *tw = nullptr;
  int *err = nullptr;
  uint16_t *abar = nullptr;
  uint32_t *acc = nullptr;
  uint16_t *ksh = nullptr;  // [1024][ksh_ld(job_cap)] rounded coefficients (tensor key switch)
  size_t job_cap = 0;
  uint64_t scratch_gen = 0;  // bumped whenever abar/acc are reallocated
  uint8_t *io_ops = nullptr;
  uint32_t *io_a = nullptr, *io_b = nullptr, *io_out = nullptr;
  size_t io_cap = 0;
  int cfg_g = 0, cfg_bps = 0;
  int cfg_ks = 0;  // key switch: 0 automatic, 1 CUDA cores, 2 tensor cores
  int cfg_xp = 0;  // external product: 0 transform (CUDA cores), 1 Toeplitz (tensor cores)
  uint16_t *tt_digits = nullptr;  // digit operand of the tensor-core external product
  size_t tt_cap = 0;              // jobs the digit operand holds
  int last_launches = 0;
  // Optional per-kernel timing: event pairs recorded around each launch on
  // the launching stream, summed by ce_profile_read.
  bool profile = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Timed { int kind; cudaEvent_t a, b; };
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> mma_ev;  // pending events of kind 3
  ce::Engine *engine = nullptr;
  // Autotuned blind-rotation shape: gates per block for measured job counts.
  std::vector<int> tune_jobs, tune_g;
};

namespace ce {

// Shared helpers of the context translation units.
ce_status cuda_error(cudaError_t e, const char *where);
ce_status ensure_job_scratch(ce_ctx *ctx, size_t jobs);
cudaEvent_t take_event(ce_ctx *ctx);
void br_shape(const ce_ctx *ctx, size_t jobs, int *G, int *blocks);
// Row stride (outputs) of the rounded-coefficient scratch for a job capacity.
inline int ksh_ld(size_t job_cap) { return int((job_cap + 16 + 7) / 8 * 8); }
// Whether a single-client key switch of n_out outputs runs on the tensor cores.
bool ks_use_tensor(const ce_ctx *ctx, size_t n_out);
void ks_shape(const ce_ctx *ctx, size_t n_out, int *tile, int *jsplit);
// Builds the client's Hankel limb sequences if missing (counted against the
// context's HBM budget).
ce_status ensure_hankel(ce_ctx *ctx, Client *cl);
void engine_destroy(Engine *e);
void engine_drop_client(Engine *e, int client);
// Records an event pair around `launch` when profiling is on (kind 0, 1, 2).
// Event pairs for the MMA launches of a tensor-core blind rotation (kind 3)
// while profiling is on, else nullptr; keep_mma_events files them.
cudaEvent_t *mma_events(ce_ctx *ctx);
void keep_mma_events(ce_ctx *ctx);
template <class F>
cudaError_t timed(ce_ctx *ctx, int kind, cudaStream_t st, F launch) {
  if (!ctx->profile) return launch();
  cudaEvent_t a = take_event(ctx), b = take_event(ctx);
  cudaEventRecord(a, st);
  cudaError_t e = launch();
  cudaEventRecord(b, st);
  ctx->timed.push_back({kind, a, b});
  return e;
}

}  // namespace ce
