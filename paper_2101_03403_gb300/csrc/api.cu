// C ABI of the library: contexts, client admission, batched gates.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ce_internal.h"
#include "launch.h"
#include "rns_arith.h"

namespace ce {

namespace {
thread_local std::string g_last_error;
constexpr uint64_t kMaxSelftestWaitNs = 2000000000ull;

}  // namespace

ce_status set_error(ce_status code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

namespace {
std::atomic<uint64_t> g_dev_allocs{0}, g_dev_frees{0};
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_dev_allocs.fetch_add(1, std::memory_order_relaxed);
  return e;
}

void dev_free(void *p) {
  if (!p) return;
  cudaFree(p);
  g_dev_frees.fetch_add(1, std::memory_order_relaxed);
}

// Per-thread factors of the two-prime transform (rns_ntt.cuh) with their
// Shoup quotients: twists (the inverse ones carry the 1/1024 scale) and the
// middle-phase twiddles.
void transform_tables(uint4 *out) {
  const uint32_t ps[2] = {rns::P<0>(), rns::P<1>()};
  const uint32_t roots[2] = {rns::Psi<0>(), rns::Psi<1>()};
  for (int q = 0; q < 2; ++q) {
    const uint32_t p = ps[q], psi = roots[q], psi_inv = rns::invm(psi, p);
    const uint32_t inv1024 = rns::invm(1024, p);
    for (int k2 = 0; k2 < 16; ++k2)
      for (int n1 = 0; n1 < 64; ++n1) {
        const uint64_t e = uint64_t(2 * k2 + 1) * n1;
        const uint32_t wf = rns::powm(psi, e, p);
        const uint32_t wi = rns::mulm(rns::powm(psi_inv, e, p), inv1024, p);
        uint4 &F = out[k2 * 64 + n1], &I = out[1024 + k2 * 64 + n1];
        (q == 0 ? F.x : F.z) = wf;
        (q == 0 ? F.y : F.w) = rns::shoup_of(wf, p);
        (q == 0 ? I.x : I.z) = wi;
        (q == 0 ? I.y : I.w) = rns::shoup_of(wi, p);
      }
    for (int a = 0; a < 8; ++a)
      for (int c = 0; c < 8; ++c) {
        const uint64_t e = uint64_t(32) * a * c;
        const uint32_t wf = rns::powm(psi, e, p), wi = rns::powm(psi_inv, e, p);
        uint4 &F = out[2048 + a * 8 + c], &I = out[2112 + a * 8 + c];
        (q == 0 ? F.x : F.z) = wf;
        (q == 0 ? F.y : F.w) = rns::shoup_of(wf, p);
        (q == 0 ? I.x : I.z) = wi;
        (q == 0 ? I.y : I.w) = rns::shoup_of(wi, p);
      }
  }
}

}  // namespace ce

using namespace ce;

#include "ctx.h"

namespace {

ce_status cuda_fail(cudaError_t e, const char *where) {
  return set_error(CE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

namespace {

// Digit operand of the tensor-core external product, sized like the job
// scratch once that form is selected.
ce_status ensure_tt_digits(ce_ctx *ctx, size_t jobs) {
  if (ctx->cfg_xp != 1 || (ctx->tt_digits && jobs <= ctx->tt_cap)) return CE_OK;
  const size_t cap = std::max(jobs, ctx->job_cap);
  dev_free(ctx->tt_digits);
  ctx->tt_digits = nullptr;
  ctx->tt_cap = 0;
  ++ctx->scratch_gen;
  if (dev_malloc(&ctx->tt_digits, blind_rotate_tc_digit_bytes(cap)) != cudaSuccess)
    return set_error(CE_ENOMEM, "digit operand allocation failed");
  ctx->tt_cap = cap;
  return CE_OK;
}

ce_status ensure_jobs(ce_ctx *ctx, size_t jobs) {
  if (jobs <= ctx->job_cap) return ensure_tt_digits(ctx, jobs);
  size_t cap = ctx->job_cap ? ctx->job_cap : 64;
  while (cap < jobs) cap *= 2;
  dev_free(ctx->abar);  // synchronises with work still using the old scratch
  dev_free(ctx->acc);
  dev_free(ctx->ksh);
  ctx->abar = nullptr;
  ctx->acc = nullptr;
  ctx->ksh = nullptr;
  ctx->job_cap = 0;
  ++ctx->scratch_gen;  // captured graphs that baked in the old pointers are stale
  cudaError_t e = dev_malloc(&ctx->abar, cap * kAbarStride * sizeof(uint16_t));
  if (e == cudaSuccess) e = dev_malloc(&ctx->acc, cap * 2 * kRingN * sizeof(uint32_t));
  // rounded coefficients of the tensor-core key switch: [1024][ksh_ld] (an
  // engine tick pads its outputs to tiles of 16 beyond its jobs)
  if (e == cudaSuccess) e = dev_malloc(&ctx->ksh, size_t(kRingN) * ksh_ld(cap) * sizeof(uint16_t));
  if (e != cudaSuccess) return set_error(CE_ENOMEM, "scratch allocation failed");
  ctx->job_cap = cap;
  return ensure_tt_digits(ctx, cap);
}

ce_status ensure_io(ce_ctx *ctx, size_t n) {
  if (n <= ctx->io_cap) return CE_OK;
  size_t cap = ctx->io_cap ? ctx->io_cap : 64;
  while (cap < n) cap *= 2;
  dev_free(ctx->io_ops);
  dev_free(ctx->io_a);
  dev_free(ctx->io_b);
  dev_free(ctx->io_out);
  ctx->io_ops = nullptr;
  ctx->io_a = ctx->io_b = ctx->io_out = nullptr;
  ctx->io_cap = 0;
  const size_t w = cap * kLweWords * sizeof(uint32_t);
  cudaError_t e = dev_malloc(&ctx->io_ops, cap);
  if (e == cudaSuccess) e = dev_malloc(&ctx->io_a, w);
  if (e == cudaSuccess) e = dev_malloc(&ctx->io_b, w);
  if (e == cudaSuccess) e = dev_malloc(&ctx->io_out, w);
  if (e != cudaSuccess) return set_error(CE_ENOMEM, "staging allocation failed");
  ctx->io_cap = cap;
  return CE_OK;
}

Client *find_client(ce_ctx *ctx, int id) {
  if (id < 0 || id >= int(ctx->clients.size()) || !ctx->clients[id].live) return nullptr;
  return &ctx->clients[id];
}

// Blind-rotation launch shape: gates per block and resident blocks per SM.
void br_config(const ce_ctx *ctx, size_t jobs, int *G, int *blocks) {
  int g = ctx->cfg_g, bps = ctx->cfg_bps;
  if (g == 0 && !ctx->tune_jobs.empty()) {
    // autotuned: the shape measured fastest at the nearest job count (log scale)
    size_t best = 0;
    double bd = 1e30;
    for (size_t i = 0; i < ctx->tune_jobs.size(); ++i) {
      const double d = std::fabs(std::log(double(jobs) + 1) - std::log(double(ctx->tune_jobs[i]) + 1));
      if (d < bd) {
        bd = d;
        best = i;
      }
    }
    g = ctx->tune_g[best];
  }
  if (g == 0) {
    if (jobs >= size_t(8) * ctx->sms) g = 4;
    else if (jobs >= size_t(2) * ctx->sms) g = 2;
    else g = 1;
  }
  if (bps == 0) bps = (g == 1) ? 2 : 1;
  const int per_block = g == 3 ? 1 : g;  // shape 3: one gate, three groups
  const size_t groups = (jobs + per_block - 1) / per_block;
  size_t b = size_t(ctx->sms) * bps;
  if (groups < b) b = groups;
  *G = g;
  *blocks = int(b);
}

void ks_config(const ce_ctx *ctx, size_t n_out, int *tile, int *jsplit) {
  int t = n_out >= 64 ? 16 : (n_out >= 4 ? 4 : 1);
  const size_t tiles = (n_out + t - 1) / t;
  size_t js = (size_t(2) * ctx->sms + tiles - 1) / tiles;
  if (js < 1) js = 1;
  if (js > 64) js = 64;
  *tile = t;
  *jsplit = int(js);
}

// Jobs -> blind rotation -> extraction/key switching on device buffers.
ce_status run_path(ce_ctx *ctx, Client *cl, int mode, const uint8_t *ops, const uint32_t *a,
                   const uint32_t *b, const uint32_t *c, uint32_t *out, size_t n,
                   cudaStream_t st) {
  const size_t jobs = mode ? 2 * n : n;
  if (n == 0) {
    ctx->last_launches = 0;
    return CE_OK;
  }
  if (jobs > size_t(1) << 30) return set_error(CE_EINVAL, "batch too large");
  ce_status s = ensure_jobs(ctx, jobs);
  if (s != CE_OK) return s;
  int launches = 0;
  cudaError_t e = ce::timed(ctx, 0, st, [&] {
    return launch_lincomb_modswitch(ops, a, b, c, ctx->abar, int(jobs), mode, ctx->err, st);
  });
  if (e != cudaSuccess) return cuda_fail(e, "lincomb_modswitch");
  ++launches;
  if (ctx->cfg_xp == 1) {
    s = ensure_hankel(ctx, cl);
    if (s != CE_OK) return s;
    const int ctas = blind_rotate_tc_ctas(ctx->sms, int(jobs));
    e = ce::timed(ctx, 1, st, [&] {
      return launch_blind_rotate_tc(cl->bsk_hankel, ctx->abar, ctx->acc, int(jobs),
                                    ctx->tt_digits, ctas, ctx->err, st, &launches,
                                    mma_events(ctx));
    });
    keep_mma_events(ctx);
    if (e != cudaSuccess) return cuda_fail(e, "blind_rotate_tc");
  } else {
    int G, blocks;
    br_config(ctx, jobs, &G, &blocks);
    e = ce::timed(ctx, 1, st, [&] {
      return launch_blind_rotate(cl->bsk, ctx->abar, ctx->acc, int(jobs), ctx->tw, ctx->err, G,
                                 blocks, st, nullptr, &launches);
    });
    if (e != cudaSuccess) return cuda_fail(e, "blind_rotate");
  }
  if (ks_use_tensor(ctx, n)) {
    int n_tile, out_tiles, ksplit;
    keyswitch_tc_shape(ctx->sms, int(n), &n_tile, &out_tiles, &ksplit);
    if (ksplit > 1) {
      e = cudaMemsetAsync(out, 0, n * kLweWords * sizeof(uint32_t), st);
      if (e != cudaSuccess) return cuda_fail(e, "memset");
    }
    e = ce::timed(ctx, 2, st, [&] {
      return launch_keyswitch_tc(ctx->acc, cl->ksk_planes, nullptr, out, int(n), mode != 0 ? 1 : 0,
                                 n_tile, out_tiles, ksplit, ctx->ksh, ksh_ld(ctx->job_cap),
                                 ctx->err, st);
    });
    ++launches;  // the rounding pass
  } else {
    int tile, jsplit;
    ks_config(ctx, n, &tile, &jsplit);
    if (jsplit > 1) {
      e = cudaMemsetAsync(out, 0, n * kLweWords * sizeof(uint32_t), st);
      if (e != cudaSuccess) return cuda_fail(e, "memset");
    }
    e = ce::timed(ctx, 2, st, [&] {
      return launch_extract_keyswitch(ctx->acc, cl->ksk, out, int(n), mode != 0, tile, jsplit, st);
    });
  }
  if (e != cudaSuccess) return cuda_fail(e, "extract_keyswitch");
  ++launches;
  ctx->last_launches = launches;
  return CE_OK;
}

}  // namespace

namespace ce {

ce_status check_device_error(ce_ctx *ctx) {
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "error flag read");
  if (h) {
    cudaMemset(ctx->err, 0, sizeof(int));
    if (h == 2) return set_error(CE_EINVAL, "a device gate opcode was out of range");
    return set_error(CE_ETIMEOUT, "a device-side wait expired (results invalid)");
  }
  return CE_OK;
}

}  // namespace ce

extern "C" const char *ce_last_error(void) { return g_last_error.c_str(); }

extern "C" void ce_device_alloc_count(uint64_t *allocations, uint64_t *frees) {
  if (allocations) *allocations = g_dev_allocs.load();
  if (frees) *frees = g_dev_frees.load();
}

extern "C" uint64_t ce_client_footprint_bytes(void) { return kClientBytes; }

extern "C" ce_status ce_create(ce_ctx **out, int device, uint64_t hbm_budget_bytes,
                               void *cuda_stream) {
  if (!out) return set_error(CE_EINVAL, "ce_create: null output");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0) return set_error(CE_ECUDA, "ce_create: no CUDA device");
  if (device < 0 || device >= count) return set_error(CE_EINVAL, "ce_create: bad device index");
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  ce_ctx *ctx = new ce_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : uint64_t(free_b) / 10 * 9;
  std::vector<uint4> tw(kTwistEntries);
  transform_tables(tw.data());
  e = dev_malloc(&ctx->tw, kTwistEntries * sizeof(uint4));
  if (e == cudaSuccess) e = dev_malloc(&ctx->err, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->tw, tw.data(), kTwistEntries * sizeof(uint4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ctx->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->order_ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ce_destroy(ctx);
    return cuda_fail(e, "ce_create");
  }
  *out = ctx;
  return CE_OK;
}

extern "C" void ce_destroy(ce_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();  // work may be in flight on callers' streams
  for (auto &c : ctx->clients) {
    dev_free(c.bsk);
    dev_free(c.ksk);
    dev_free(c.ksk_planes);
    dev_free(c.bsk_coef);
    dev_free(c.bsk_hankel);
  }
  dev_free(ctx->tw);
  dev_free(ctx->tt_digits);
  dev_free(ctx->ksh);
  dev_free(ctx->err);
  dev_free(ctx->abar);
  dev_free(ctx->acc);
  dev_free(ctx->io_ops);
  dev_free(ctx->io_a);
  dev_free(ctx->io_b);
  dev_free(ctx->io_out);
  engine_destroy(ctx->engine);
  ctx->engine = nullptr;
  for (auto &t : ctx->timed) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->order_ev) cudaEventDestroy(ctx->order_ev);
  delete ctx;
}

extern "C" ce_status ce_client_admit(ce_ctx *ctx, const void *cloud_key, size_t bytes,
                                     int *client_id) {
  if (!ctx || !cloud_key || !client_id) return set_error(CE_EINVAL, "ce_client_admit: null arg");
  const uint32_t *w = static_cast<const uint32_t *>(cloud_key);
  if (bytes != CE_CLOUD_BYTES || w[0] != 0x4B434543u || w[1] != 1u)
    return set_error(CE_EINVAL, "ce_client_admit: not a cloud key");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  if (ctx->used + kClientBytes > ctx->budget)
    return set_error(CE_EADMIT, "ce_client_admit: over the HBM budget");
  cudaSetDevice(ctx->device);
  Client cl;
  uint32_t *coef = nullptr;
  cudaError_t e = dev_malloc(&cl.bsk, kBskNttBytes);
  if (e == cudaSuccess) e = dev_malloc(&cl.ksk, kKskDevBytes);
  if (e == cudaSuccess) e = dev_malloc(&cl.ksk_planes, kKsPlaneBytes);
  if (e == cudaSuccess) e = dev_malloc(&coef, size_t(CE_BSK_WORDS) * 4);
  if (e != cudaSuccess) {
    dev_free(cl.bsk);
    dev_free(cl.ksk);
    dev_free(cl.ksk_planes);
    dev_free(coef);
    return set_error(CE_ENOMEM, "ce_client_admit: device allocation failed");
  }
  const uint32_t *bsk = w + 2;
  const uint32_t *ksk = bsk + CE_BSK_WORDS;
  // Key-switching key rows v = 1..3, padded to 512 words.
  std::vector<uint32_t> kd(kKskDevWords, 0u);
  for (int j = 0; j < kRingN; ++j)
    for (int q = 0; q < kKsT; ++q)
      for (int v = 1; v < kKsBase; ++v) {
        const uint32_t *src = ksk + ((size_t(j) * kKsT + q) * kKsBase + v) * kLweWords;
        uint32_t *dst = kd.data() + ((size_t(j) * kKsT + q) * 3 + (v - 1)) * kKskRow;
        std::memcpy(dst, src, kLweWords * sizeof(uint32_t));
      }
  cudaStream_t st = ctx->stream;
  e = cudaMemcpyAsync(coef, bsk, size_t(CE_BSK_WORDS) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cl.ksk, kd.data(), kKskDevBytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_bsk_to_transform(coef, cl.bsk, ctx->tw, st);
  if (e == cudaSuccess) e = launch_ksk_to_planes(cl.ksk, cl.ksk_planes, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    dev_free(cl.bsk);
    dev_free(cl.ksk);
    dev_free(cl.ksk_planes);
    dev_free(coef);
    return cuda_fail(e, "ce_client_admit");
  }
  cl.bsk_coef = coef;
  cl.live = true;
  int id = -1;
  for (size_t i = 0; i < ctx->clients.size(); ++i)
    if (!ctx->clients[i].live) {
      id = int(i);
      break;
    }
  {
    std::lock_guard<std::mutex> cl_lock(ctx->clients_mu);
    if (id < 0) {
      id = int(ctx->clients.size());
      ctx->clients.push_back(cl);
    } else {
      ctx->clients[id] = cl;
    }
  }
  ctx->used += kClientBytes;
  *client_id = id;
  return CE_OK;
}

extern "C" ce_status ce_client_evict(ce_ctx *ctx, int client_id) {
  if (!ctx) return set_error(CE_EINVAL, "ce_client_evict: null context");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  std::lock_guard<std::mutex> cl_lock(ctx->clients_mu);
  Client *cl = find_client(ctx, client_id);
  if (!cl) return set_error(CE_ENOTFOUND, "ce_client_evict: unknown client");
  for (ce_server *s : ctx->servers)
    if (server_client_busy(s, client_id))
      return set_error(CE_EINVAL, "ce_client_evict: the client has requests queued or running "
                                  "on a serving loop");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();  // its keys may be in use on any stream
  engine_drop_client(ctx->engine, client_id);
  dev_free(cl->bsk);
  dev_free(cl->ksk);
  dev_free(cl->ksk_planes);
  dev_free(cl->bsk_coef);
  if (cl->bsk_hankel) {
    dev_free(cl->bsk_hankel);
    ctx->used -= blind_rotate_tc_key_bytes();
  }
  *cl = Client();
  ctx->used -= kClientBytes;
  return CE_OK;
}

extern "C" ce_status ce_gates_batch_device(ce_ctx *ctx, int client, const uint8_t *d_ops,
                                           const uint32_t *d_a, const uint32_t *d_b,
                                           uint32_t *d_out, size_t n, void *cuda_stream) {
  if (!ctx) return set_error(CE_EINVAL, "ce_gates_batch_device: null context");
  if (n && (!d_ops || !d_a || !d_b || !d_out))
    return set_error(CE_EINVAL, "ce_gates_batch_device: null buffer");
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  CtxWork work(ctx, st);
  Client *cl = find_client(ctx, client);
  if (!cl) return set_error(CE_ENOTFOUND, "ce_gates_batch_device: unknown client");
  return run_path(ctx, cl, 0, d_ops, d_a, d_b, nullptr, d_out, n, st);
}

extern "C" ce_status ce_mux_batch_device(ce_ctx *ctx, int client, const uint32_t *d_a,
                                         const uint32_t *d_b, const uint32_t *d_c,
                                         uint32_t *d_out, size_t n, void *cuda_stream) {
  if (!ctx) return set_error(CE_EINVAL, "ce_mux_batch_device: null context");
  if (n && (!d_a || !d_b || !d_c || !d_out))
    return set_error(CE_EINVAL, "ce_mux_batch_device: null buffer");
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  CtxWork work(ctx, st);
  Client *cl = find_client(ctx, client);
  if (!cl) return set_error(CE_ENOTFOUND, "ce_mux_batch_device: unknown client");
  return run_path(ctx, cl, 1, nullptr, d_a, d_b, d_c, d_out, n, st);
}

extern "C" ce_status ce_gates_batch(ce_ctx *ctx, int client, const uint8_t *ops,
                                    const ce_lwe *a, const ce_lwe *b, ce_lwe *out, size_t n) {
  if (!ctx) return set_error(CE_EINVAL, "ce_gates_batch: null context");
  if (n == 0) return CE_OK;
  if (!ops || !a || !b || !out) return set_error(CE_EINVAL, "ce_gates_batch: null buffer");
  for (size_t i = 0; i < n; ++i)
    if (ops[i] > CE_ORYN) return set_error(CE_EINVAL, "ce_gates_batch: bad gate opcode");
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  CtxWork work(ctx, st);
  Client *cl = find_client(ctx, client);
  if (!cl) return set_error(CE_ENOTFOUND, "ce_gates_batch: unknown client");
  ce_status s = ensure_io(ctx, n);
  if (s != CE_OK) return s;
  const size_t w = n * kLweWords * sizeof(uint32_t);
  cudaError_t e = cudaMemcpyAsync(ctx->io_ops, ops, n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->io_a, a, w, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->io_b, b, w, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "ce_gates_batch upload");
  s = run_path(ctx, cl, 0, ctx->io_ops, ctx->io_a, ctx->io_b, nullptr, ctx->io_out, n, st);
  if (s != CE_OK) return s;
  e = cudaMemcpyAsync(out, ctx->io_out, w, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "ce_gates_batch");
  return check_device_error(ctx);
}

extern "C" ce_status ce_gate(ce_ctx *ctx, int client, ce_gate_op op, const ce_lwe *a,
                             const ce_lwe *b, ce_lwe *out) {
  const uint8_t o = static_cast<uint8_t>(op);
  if (int(op) < 0 || int(op) > CE_ORYN) return set_error(CE_EINVAL, "ce_gate: bad opcode");
  return ce_gates_batch(ctx, client, &o, a, b, out, 1);
}

extern "C" ce_status ce_negacyclic_mul_device(ce_ctx *ctx, const int16_t *d_d,
                                              const uint32_t *d_k, uint32_t *d_out, size_t n,
                                              void *cuda_stream) {
  if (!ctx) return set_error(CE_EINVAL, "ce_negacyclic_mul_device: null context");
  if (n && (!d_d || !d_k || !d_out))
    return set_error(CE_EINVAL, "ce_negacyclic_mul_device: null buffer");
  if (n > (size_t(1) << 28)) return set_error(CE_EINVAL, "ce_negacyclic_mul_device: n too large");
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  cudaError_t e = launch_negacyclic_mul(d_d, d_k, d_out, int(n), ctx->tw, st);
  if (e != cudaSuccess) return cuda_fail(e, "negacyclic_mul");
  return CE_OK;
}

extern "C" ce_status ce_blind_rotate_plan(int n_jobs, int gates_per_block, int blocks,
                                          int *out) {
  if (!out || n_jobs < 0 || gates_per_block < 1 || gates_per_block > 4 || blocks < 1)
    return set_error(CE_EINVAL, "ce_blind_rotate_plan: bad arguments");
  const ce::BrSplit s = ce::blind_rotate_split(n_jobs, gates_per_block, blocks);
  out[0] = s.main_jobs;
  out[1] = s.tail_jobs;
  out[2] = s.tail_G;
  out[3] = s.tail_blocks;
  return CE_OK;
}

extern "C" ce_status ce_set_blind_rotate_config(ce_ctx *ctx, int gates_per_block,
                                                int blocks_per_sm) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_blind_rotate_config: null context");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  if (gates_per_block < 0 || gates_per_block > 4)
    return set_error(CE_EINVAL, "gates_per_block must be 0 (auto), 1, 2, 3 (one gate, three "
                                "groups) or 4");
  const int max_bps = gates_per_block == 1 ? 2 : 1;
  if (blocks_per_sm < 0 || (gates_per_block && blocks_per_sm > max_bps))
    return set_error(CE_EINVAL, "blocks_per_sm exceeds what shared memory allows");
  ctx->cfg_g = gates_per_block;
  ctx->cfg_bps = blocks_per_sm;
  return CE_OK;
}

extern "C" ce_status ce_set_keyswitch_config(ce_ctx *ctx, int engine) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_keyswitch_config: null context");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  if (engine < 0 || engine > 2)
    return set_error(CE_EINVAL, "key-switch engine must be 0 (auto), 1 (CUDA cores) or 2 "
                                "(tensor cores)");
  ctx->cfg_ks = engine;
  return CE_OK;
}

extern "C" ce_status ce_set_external_product_form(ce_ctx *ctx, int form) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_external_product_form: null context");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  if (form < 0 || form > 1)
    return set_error(CE_EINVAL, "external-product form must be 0 (transform, CUDA cores) or 1 "
                                "(Toeplitz, tensor cores)");
  ctx->cfg_xp = form;
  return CE_OK;
}

extern "C" int ce_last_launch_count(ce_ctx *ctx) { return ctx ? ctx->last_launches : 0; }

extern "C" ce_status ce_synchronize(ce_ctx *ctx) {
  if (!ctx) return set_error(CE_EINVAL, "ce_synchronize: null context");
  cudaError_t e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "ce_synchronize");
  return check_device_error(ctx);
}

extern "C" ce_status ce_selftest_device_wait(ce_ctx *ctx, uint64_t limit_ns) {
  if (!ctx) return set_error(CE_EINVAL, "ce_selftest_device_wait: null context");
  if (limit_ns < 1000 || limit_ns > kMaxSelftestWaitNs)
    return set_error(CE_EINVAL, "ce_selftest_device_wait: limit must lie in [1 us, 2 s]");
  cudaSetDevice(ctx->device);
  cudaError_t e = launch_wait_selftest(limit_ns, ctx->err, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ce_selftest_device_wait");
  return CE_OK;
}

extern "C" ce_status ce_probe_int_pipes(ce_ctx *ctx, double *lane_ops_per_clock) {
  if (!ctx || !lane_ops_per_clock) return set_error(CE_EINVAL, "ce_probe_int_pipes: bad argument");
  cudaSetDevice(ctx->device);
  CtxWork work(ctx, ctx->stream);
  // one 512-thread block per SM (16 warps, eight independent chains each)
  const int blocks = ctx->sms, iters = 4096, threads = 512;
  uint32_t *sink = nullptr;
  long long *cyc = nullptr;
  int *smid = nullptr;
  cudaError_t e = dev_malloc(&sink, size_t(blocks) * threads * sizeof(uint32_t));
  if (e == cudaSuccess) e = dev_malloc(&cyc, size_t(blocks) * sizeof(long long));
  if (e == cudaSuccess) e = dev_malloc(&smid, size_t(blocks) * sizeof(int));
  std::vector<long long> h(blocks);
  std::vector<int> hs(blocks);
  for (int kind = 0; kind < 3 && e == cudaSuccess; ++kind) {
    // the first launch of each kind warms up; the second is measured
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
      e = launch_int_pipe_probe(kind, blocks, threads, iters, sink, cyc, smid, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(hs.data(), smid, blocks * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      // per SM: the operations of its blocks over the longest of their times
      std::vector<double> ops(1024, 0.0), span(1024, 0.0);
      for (int b = 0; b < blocks; ++b) {
        const int id = hs[b] & 1023;
        ops[id] += double(threads) * 8.0 * iters;
        span[id] = std::max(span[id], double(h[b]));
      }
      double sum = 0;
      int used = 0;
      for (int id = 0; id < 1024; ++id)
        if (span[id] > 0) {
          sum += ops[id] / span[id];
          ++used;
        }
      lane_ops_per_clock[kind] = used ? sum / used : 0.0;
    }
  }
  dev_free(sink);
  dev_free(cyc);
  dev_free(smid);
  if (e != cudaSuccess) return cuda_fail(e, "ce_probe_int_pipes");
  return CE_OK;
}

extern "C" ce_status ce_profile_enable(ce_ctx *ctx, int on) {
  if (!ctx) return set_error(CE_EINVAL, "ce_profile_enable: null context");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  ctx->profile = on != 0;
  return CE_OK;
}

extern "C" ce_status ce_profile_read(ce_ctx *ctx, double *ms, int *launches, int kinds) {
  if (!ctx || !ms || !launches || kinds <= 0)
    return set_error(CE_EINVAL, "ce_profile_read: bad argument");
  std::lock_guard<std::recursive_mutex> lock(ctx->mu);
  for (int k = 0; k < kinds; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto &t : ctx->timed) {
    cudaError_t e = cudaEventSynchronize(t.b);
    if (e != cudaSuccess) return cuda_fail(e, "ce_profile_read");
    float f = 0.f;
    cudaEventElapsedTime(&f, t.a, t.b);
    if (t.kind < kinds) {
      ms[t.kind] += f;
      launches[t.kind] += 1;
    }
    ctx->ev_pool.push_back(t.a);
    ctx->ev_pool.push_back(t.b);
  }
  ctx->timed.clear();
  return CE_OK;
}

namespace ce {

// Keys and launch shapes of the gate path for entry points defined in other
// translation units.  Allocates nothing.
ce_status gate_path_resources(ce_ctx *ctx, int client, GatePathResources *out) {
  if (!ctx || !out) return set_error(CE_EINVAL, "null context");
  Client *cl = find_client(ctx, client);
  if (!cl) return set_error(CE_ENOTFOUND, "unknown client");
  out->bsk = cl->bsk;
  out->ksk = cl->ksk;
  out->tw = ctx->tw;
  out->err = ctx->err;
  out->device = ctx->device;
  out->stream = ctx->stream;
  return CE_OK;
}

void gate_path_shape(const ce_ctx *ctx, size_t jobs, size_t n_out, int *G, int *blocks,
                     int *tile, int *jsplit) {
  br_config(ctx, jobs, G, blocks);
  ks_config(ctx, n_out, tile, jsplit);
}

}  // namespace ce

namespace ce {

ce_status cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }
ce_status ensure_job_scratch(ce_ctx *ctx, size_t jobs) { return ensure_jobs(ctx, jobs); }
void br_shape(const ce_ctx *ctx, size_t jobs, int *G, int *blocks) { br_config(ctx, jobs, G, blocks); }
// Tensor cores from 32 outputs (automatic): below that the CUDA-core kernel's
// j-split keeps more SMs busy for the few outputs.
bool ks_use_tensor(const ce_ctx *ctx, size_t n_out) {
  if (ctx->cfg_ks == 1) return false;
  if (ctx->cfg_ks == 2) return n_out > 0;
  return n_out >= 32;
}
void ks_shape(const ce_ctx *ctx, size_t n_out, int *tile, int *jsplit) {
  ks_config(ctx, n_out, tile, jsplit);
}
ce_status ensure_hankel(ce_ctx *ctx, Client *cl) {
  if (cl->bsk_hankel) return CE_OK;
  const uint64_t bytes = blind_rotate_tc_key_bytes();
  if (ctx->used + bytes > ctx->budget)
    return set_error(CE_EADMIT, "tensor-core external product: key over the HBM budget");
  if (dev_malloc(&cl->bsk_hankel, bytes) != cudaSuccess) {
    cl->bsk_hankel = nullptr;
    return set_error(CE_ENOMEM, "tensor-core external product: key allocation failed");
  }
  cudaError_t e = launch_bsk_to_hankel(cl->bsk_coef, cl->bsk_hankel, ctx->stream);
  if (e == cudaSuccess) e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    dev_free(cl->bsk_hankel);
    cl->bsk_hankel = nullptr;
    return cuda_error(e, "bsk_to_hankel");
  }
  ctx->used += bytes;
  return CE_OK;
}
cudaEvent_t *mma_events(ce_ctx *ctx) {
  if (!ctx->profile) return nullptr;
  ctx->mma_ev.resize(2 * kLweN);
  for (auto &e : ctx->mma_ev) e = take_event(ctx);
  return ctx->mma_ev.data();
}
void keep_mma_events(ce_ctx *ctx) {
  for (size_t i = 0; i + 1 < ctx->mma_ev.size(); i += 2)
    ctx->timed.push_back({3, ctx->mma_ev[i], ctx->mma_ev[i + 1]});
  ctx->mma_ev.clear();
}
cudaEvent_t take_event(ce_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace ce

// Autotuner: times the blind-rotation kernel with 1, 2 and 4 gates per block
// at a ladder of job counts (on the client's key, synthetic inputs) and keeps
// the fastest shape per count; later launches use the nearest measured count.
extern "C" ce_status ce_autotune(ce_ctx *ctx, int client, int *out_jobs, int *out_g, int cap,
                                 int *count) {
  if (!ctx) return set_error(CE_EINVAL, "ce_autotune: null context");
  CtxWork work(ctx, ctx->stream);
  Client *cl = find_client(ctx, client);
  if (!cl) return set_error(CE_ENOTFOUND, "ce_autotune: unknown client");
  const int ladder[] = {1, 8, 38, 76, 152, 304, 608, 1216, 2432, 4864, 9728};
  const int nl = int(sizeof(ladder) / sizeof(ladder[0]));
  ce_status s = ensure_jobs(ctx, size_t(ladder[nl - 1]));
  if (s != CE_OK) return s;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  // synthetic modulus-switched inputs (uniform in [0, 2048))
  std::vector<uint16_t> h(size_t(ladder[nl - 1]) * kAbarStride);
  uint32_t x = 0x9E3779B9u;
  for (auto &v : h) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    v = uint16_t(x & 2047u);
  }
  cudaError_t e = cudaMemcpyAsync(ctx->abar, h.data(), h.size() * sizeof(uint16_t),
                                  cudaMemcpyHostToDevice, st);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  std::vector<int> tj, tg;
  const int saved_g = ctx->cfg_g, saved_bps = ctx->cfg_bps;
  for (int i = 0; i < nl && e == cudaSuccess; ++i) {
    float best = 1e30f;
    int best_g = 1;
    for (int g : {1, 2, 3, 4}) {
      ctx->cfg_g = g;
      ctx->cfg_bps = 0;
      int G, blocks;
      br_config(ctx, size_t(ladder[i]), &G, &blocks);
      float ms = 0.f;
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // first run warms up
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess)
          e = launch_blind_rotate(cl->bsk, ctx->abar, ctx->acc, ladder[i], ctx->tw, ctx->err, G,
                                  blocks, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
      }
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_g = g;
      }
    }
    tj.push_back(ladder[i]);
    tg.push_back(best_g);
  }
  ctx->cfg_g = saved_g;
  ctx->cfg_bps = saved_bps;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return cuda_fail(e, "ce_autotune");
  ctx->tune_jobs = tj;
  ctx->tune_g = tg;
  if (count) *count = int(tj.size());
  for (int i = 0; i < int(tj.size()) && i < cap; ++i) {
    if (out_jobs) out_jobs[i] = tj[i];
    if (out_g) out_g[i] = tg[i];
  }
  return check_device_error(ctx);
}
