// Gate batches that allocate no device memory.
//
// ce_gates_batch_device grows its scratch (the modulus-switched inputs and
// the blind-rotation accumulators, 10 KB per gate) with cudaMalloc on
// demand.  Some callers cannot let that happen: a serving loop that keeps
// other streams busy cannot afford cudaMalloc's implicit device-wide
// synchronisation, and a process whose device memory is reserved up front by
// another allocator (a framework's caching allocator, a fixed budget) has
// nothing left to give.  ce_gates_batch_device_noalloc runs the same three
// kernels on a scratch area that is part of this library's image: a
// file-scope __device__ array sized for kNoallocMaxGates gates, which every
// GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ce_internal.h"
#include "ctx.h"
#include "launch.h"

namespace {

using namespace ce;

constexpr size_t kNoallocMaxGates = 256;
constexpr size_t kAbarBytes = kNoallocMaxGates * kAbarStride * sizeof(uint16_t);  // 256 KiB
constexpr size_t kAccBytes = kNoallocMaxGates * 2 * kRingN * sizeof(uint32_t);    // 2 MiB

// The scratch area.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kAbarBytes + kAccBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch area on `device` (which must be current),
// looked up once per device and cached.
ce_status scratch_address(int device, void **addr) {
  if (device < 0 || device >= kMaxDevices)
    return set_error(CE_EINVAL, "ce_gates_batch_device_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(CE_ECUDA, std::string("ce_gates_batch_device_noalloc: "
                                             "cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[device] = p;
  }
  *addr = g_scratch_addr[device];
  return CE_OK;
}

ce_status fail(cudaError_t e, const char *what) {
  return set_error(CE_ECUDA, std::string("ce_gates_batch_device_noalloc: ") + what + ": " +
                                 cudaGetErrorString(e));
}

}  // namespace

extern "C" ce_status ce_gates_batch_device_noalloc(ce_ctx *ctx, int client, const uint8_t *d_ops,
                                                   const uint32_t *d_a, const uint32_t *d_b,
                                                   uint32_t *d_out, size_t n,
                                                   void *cuda_stream) {
  if (!ctx) return set_error(CE_EINVAL, "ce_gates_batch_device_noalloc: null context");
  if (n > kNoallocMaxGates)
    return set_error(CE_EINVAL, "ce_gates_batch_device_noalloc: at most 256 gates per call");
  if (n && (!d_ops || !d_a || !d_b || !d_out))
    return set_error(CE_EINVAL, "ce_gates_batch_device_noalloc: null buffer");
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  CtxWork work(ctx, st);  // context lock; ordered after the context's earlier work
  GatePathResources res;
  ce_status s = gate_path_resources(ctx, client, &res);
  if (s != CE_OK) return s;
  if (n == 0) {
    ctx->last_launches = 0;
    return CE_OK;
  }

  int current = -1;
  cudaError_t e = cudaGetDevice(&current);
  if (e != cudaSuccess) return fail(e, "cudaGetDevice");
  if (current != res.device) {
    e = cudaSetDevice(res.device);
    if (e != cudaSuccess) return fail(e, "cudaSetDevice");
  }
  void *base = nullptr;
  s = scratch_address(res.device, &base);
  if (s == CE_OK) {
    uint16_t *abar = static_cast<uint16_t *>(base);
    uint32_t *acc = reinterpret_cast<uint32_t *>(static_cast<unsigned char *>(base) + kAbarBytes);
    int G, blocks, tile, jsplit;
    gate_path_shape(ctx, n, n, &G, &blocks, &tile, &jsplit);
    int br_launches = 0;
    // the same kinds as the allocating path, so per-kernel timing sees them
    e = timed(ctx, 0, st, [&] {
      return launch_lincomb_modswitch(d_ops, d_a, d_b, nullptr, abar, int(n), 0, res.err, st);
    });
    if (e != cudaSuccess) {
      s = fail(e, "lincomb_modswitch");
    } else if ((e = timed(ctx, 1, st, [&] {
                  return launch_blind_rotate(res.bsk, abar, acc, int(n), res.tw, res.err, G,
                                             blocks, st, nullptr, &br_launches);
                })) != cudaSuccess) {
      s = fail(e, "blind_rotate");
    } else if (jsplit > 1 &&
               (e = cudaMemsetAsync(d_out, 0, n * kLweWords * sizeof(uint32_t), st)) !=
                   cudaSuccess) {
      s = fail(e, "memset of the output");
    } else if ((e = timed(ctx, 2, st, [&] {
                  return launch_extract_keyswitch(acc, res.ksk, d_out, int(n), false, tile,
                                                  jsplit, st);
                })) != cudaSuccess) {
      s = fail(e, "extract_keyswitch");
    } else {
      ctx->last_launches = 2 + br_launches;
    }
  }
  if (current != res.device) cudaSetDevice(current);
  return s;
}
