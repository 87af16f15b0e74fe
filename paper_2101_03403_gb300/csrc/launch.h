// Host-side launchers of the library's kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "ce_internal.h"

namespace ce {

cudaError_t launch_lincomb_modswitch(const uint8_t *ops, const uint32_t *a, const uint32_t *b,
                                     const uint32_t *c, uint16_t *abar, int n_jobs, int mode,
                                     int *err, cudaStream_t st);
cudaError_t launch_blind_rotate(const uint64_t *bsk, const uint16_t *abar, uint32_t *acc,
                                int n_jobs, const uint64_t *tw, int *err, int gates_per_block,
                                int blocks, cudaStream_t st);
size_t blind_rotate_smem_bytes(int gates_per_block);
cudaError_t launch_extract_keyswitch(const uint32_t *acc, const uint32_t *ksk, uint32_t *out,
                                     int n_out, bool mux, int tile, int jsplit, cudaStream_t st);
cudaError_t launch_bsk_to_transform(const uint32_t *bsk, uint64_t *out, const uint64_t *tw,
                                    cudaStream_t st);
cudaError_t launch_negacyclic_mul(const int16_t *d, const uint32_t *k, uint32_t *out, int n,
                                  const uint64_t *tw, cudaStream_t st);

struct GatePathResources {
  const uint64_t *bsk;   // transform-domain bootstrapping key of the client
  const uint32_t *ksk;   // device key-switching key of the client
  const uint64_t *tw;    // twist tables
  int *err;              // device error flag of the context
  int device;
  cudaStream_t stream;
};

// Forward twist table psi^((2 k2 + 1) n1) at [k2 * 64 + n1] and the inverse
// table psi^(-(2 k2 + 1) n1) / 1024 at [1024 + k2 * 64 + n1].
void transform_tables(uint64_t *host_out /* 2048 words */);

}  // namespace ce

struct ce_ctx;
namespace ce {
ce_status gate_path_resources(ce_ctx *ctx, int client, GatePathResources *out);
void gate_path_shape(const ce_ctx *ctx, size_t jobs, size_t n_out, int *G, int *blocks,
                     int *tile, int *jsplit);
}  // namespace ce
