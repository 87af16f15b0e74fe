// The context object behind the C ABI (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
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

struct ce_server;

struct ce_ctx {
  // Host threads that enqueue work on the context (API calls and the worker
  // of a serving loop) take this lock; their GPU work is ordered through
  // order_ev (see ce::CtxWork).
  std::recursive_mutex mu;
  cudaEvent_t order_ev = nullptr;
  bool order_recorded = false;
  std::vector<ce_server *> servers;  // live serving loops on this context
  // Guards the structure of `clients` for readers that do not take `mu`
  // (request submission); writers hold both.
  std::mutex clients_mu;
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
  bool per_gate = false;  // engine levels as one launch per gate and step (comparison mode)
  bool fast_circuits = false;  // instructions ADD / SUB / MUL on ADD_MUX / SUB_MUX / MUL_TREE
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
// One call that enqueues GPU work on `st` using the context's shared state
// (scratch, engine arena, keys): holds the context lock for the call and
// orders the call's GPU work after the previous such call's, whatever stream
// that one used (a serving loop's worker enqueues on its own stream).  While
// `st` is being captured into a CUDA graph no ordering is added (an event
// recorded outside a capture cannot be waited on inside it).
class CtxWork {
 public:
  CtxWork(ce_ctx *c, cudaStream_t st) : ctx_(c), lock_(c->mu), st_(st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    capturing_ = cs != cudaStreamCaptureStatusNone;
    if (!capturing_ && ctx_->order_ev && ctx_->order_recorded)
      cudaStreamWaitEvent(st, ctx_->order_ev, 0);
  }
  ~CtxWork() {
    if (capturing_ || !ctx_->order_ev) return;
    if (cudaEventRecord(ctx_->order_ev, st_) == cudaSuccess) ctx_->order_recorded = true;
  }
  CtxWork(const CtxWork &) = delete;
  CtxWork &operator=(const CtxWork &) = delete;

 private:
  ce_ctx *ctx_;
  std::lock_guard<std::recursive_mutex> lock_;
  cudaStream_t st_;
  bool capturing_ = false;
};

// Reads and clears the context's device error flag (CE_ETIMEOUT for an
// expired bounded wait, CE_EINVAL for a bad device opcode).
ce_status check_device_error(ce_ctx *ctx);

// True while a serving loop on the context has a request of `client`
// queued or in flight (serve.cu).
bool server_client_busy(ce_server *s, int client);

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
