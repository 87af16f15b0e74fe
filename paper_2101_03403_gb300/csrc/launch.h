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
// grp_bsk (optional): per gate-group key (group g = gates [g*G, g*G+G);
// G = 1 for the latency shape 3).  A batch whose groups leave a part-filled
// last round over the blocks runs as two launches: the whole rounds in the
// given shape, then the remaining gates in a shape with fewer gates per
// block (blind_rotate_split; the tail's keys are looked up in the same
// grp_bsk).  launches (optional) is incremented per kernel launched.
cudaError_t launch_blind_rotate(const uint64_t *bsk, const uint16_t *abar, uint32_t *acc,
                                int n_jobs, const uint4 *tw, int *err, int gates_per_block,
                                int blocks, cudaStream_t st,
                                const uint64_t *const *grp_bsk = nullptr, int *launches = nullptr);
struct BrSplit {
  int main_jobs, tail_jobs, tail_G, tail_blocks;
};
BrSplit blind_rotate_split(int n_jobs, int gates_per_block, int blocks);
size_t blind_rotate_smem_bytes(int gates_per_block);
cudaError_t launch_extract_keyswitch(const uint32_t *acc, const uint32_t *ksk, uint32_t *out,
                                     int n_out, bool mux, int tile, int jsplit, cudaStream_t st);
// Netlist-engine descriptors.  A ciphertext slot of the engine's arena is
// kSlotWords uint32 (a[500], b, padding).
struct GateJob {
  uint32_t a, b;        // arena slots of the two inputs
  uint8_t op;           // 0..9 gate, 10/11 MUX halves
  uint8_t neg_a, neg_b;
  uint8_t pad;
};
struct GateOut {
  int32_t job1, job2;   // accumulators (job2 >= 0: MUX, adds (0, +1/8))
  uint32_t slot;        // arena slot written
  uint32_t pad;
};
cudaError_t launch_lincomb_gather(const GateJob *jobs, const uint32_t *arena, uint16_t *abar,
                                  int n_jobs, int *err, cudaStream_t st);
// mode 0: packed outputs, one job each; 1: MUX pairs; 2: descriptors to the arena.
cudaError_t launch_extract_keyswitch_ex(const uint32_t *acc, const uint32_t *ksk,
                                        const uint32_t *const *tile_ksk, const GateOut *outs,
                                        uint32_t *out, int n_out, int mode, int tile, int jsplit,
                                        cudaStream_t st);
cudaError_t launch_zero_slots(const GateOut *outs, uint32_t *arena, int n_out, cudaStream_t st);
cudaError_t launch_bsk_to_transform(const uint32_t *bsk, uint64_t *out, const uint4 *tw,
                                    cudaStream_t st);
cudaError_t launch_negacyclic_mul(const int16_t *d, const uint32_t *k, uint32_t *out, int n,
                                  const uint4 *tw, cudaStream_t st);

// Key switching on the tensor cores (keyswitch_tc.cu): the key-switching
// key as three fp16 limb planes (admission), and the fused extraction + key
// switch as a one-hot x key matrix product.  mode as for
// launch_extract_keyswitch_ex (0 packed, 1 MUX pairs, 2 descriptors).  With
// ksplit > 1 the outputs must be zero and are accumulated atomically.
size_t keyswitch_tc_plane_bytes();
cudaError_t launch_ksk_to_planes(const uint32_t *ksk, uint16_t *planes, cudaStream_t st);
void keyswitch_tc_shape(int sms, int n_out, int *n_tile, int *out_tiles, int *ksplit);
// h: scratch of [1024][ldh] uint16 (ldh >= n_out) for the rounded coefficients.
cudaError_t launch_keyswitch_tc(const uint32_t *acc, const uint16_t *planes, const GateOut *outs,
                                uint32_t *out, int n_out, int mode, int n_tile, int out_tiles,
                                int ksplit, uint16_t *h, int ldh, int *err, cudaStream_t st);

// Blind rotation with the Toeplitz external product on the tensor cores
// (blind_rotate_tc.cu).  hankel: the client's key as Hankel limb sequences
// (blind_rotate_tc_key_bytes, built by launch_bsk_to_hankel from the
// coefficient key); digits: scratch of blind_rotate_tc_digit_bytes(n_jobs).
// Launches 1 + 2 n kernels; ACC layout as launch_blind_rotate.  ctas: the
// MMA launches' grid, one stream-K range each (blind_rotate_tc_ctas: one per
// SM, fewer only for a step with fewer units than SMs).  mma_ev (optional,
// 2 n events): recorded before and after each step's MMA launch.
size_t blind_rotate_tc_key_bytes();
size_t blind_rotate_tc_digit_bytes(size_t n_jobs);
cudaError_t launch_bsk_to_hankel(const uint32_t *bsk, uint16_t *hankel, cudaStream_t st);
int blind_rotate_tc_ctas(int sms, int n_jobs);
cudaError_t launch_blind_rotate_tc(const uint16_t *hankel, const uint16_t *abar, uint32_t *acc,
                                   int n_jobs, uint16_t *digits, int ctas, int *err,
                                   cudaStream_t st, int *launches,
                                   cudaEvent_t *mma_ev = nullptr);

// Integer multiply-add pipe probe (measurement): `blocks` blocks of
// `threads` threads (at most 512), each timing iters x 8 chained operations
// of one kind (0 32-bit multiply-add, 1 high-half multiply, 2 64-bit-result
// multiply-add) with the SM clock into cycles[block], its SM into smid[block].
cudaError_t launch_int_pipe_probe(int kind, int blocks, int threads, int iters, uint32_t *sink,
                                  long long *cycles, int *smid, cudaStream_t st);

// Failure-detection self-test: a one-thread bounded wait on a barrier that
// nothing completes, with the given limit (sets *err on expiry).
cudaError_t launch_wait_selftest(uint64_t limit_ns, int *err, cudaStream_t st);

struct GatePathResources {
  const uint64_t *bsk;   // transform-domain bootstrapping key of the client
  const uint32_t *ksk;   // device key-switching key of the client
  const uint4 *tw;       // twist tables
  int *err;              // device error flag of the context
  int device;
  cudaStream_t stream;
};

// Factor table of the two-prime transform, one uint4 {w0, w0', w1, w1'} per
// entry (residue mod p_q and its Shoup quotient): forward twist
// psi_q^((2 k2 + 1) n1) at [k2 * 64 + n1], inverse twist
// psi_q^(-(2 k2 + 1) n1) / 1024 at [1024 + k2 * 64 + n1], middle-phase
// twiddles psi_q^(32 a c) at [2048 + a * 8 + c] and psi_q^(-32 a c) at
// [2112 + a * 8 + c].
constexpr size_t kTwistEntries = 2176;
void transform_tables(uint4 *host_out /* kTwistEntries */);

}  // namespace ce

struct ce_ctx;
namespace ce {
ce_status gate_path_resources(ce_ctx *ctx, int client, GatePathResources *out);
void gate_path_shape(const ce_ctx *ctx, size_t jobs, size_t n_out, int *G, int *blocks,
                     int *tile, int *jsplit);
}  // namespace ce
