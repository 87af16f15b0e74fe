// Level-synchronous netlist engine: functional units and instruction
// programs over bootstrapped gates, batched across instructions and clients.
//
// The paper's emulator evaluates each functional unit with OpenMP sections,
// one thread per gate, serialised past its 48 cores (§5).  Here every
// in-flight unit instance (an instruction of some client) contributes the
// gates of its next level to one "tick": a single batched launch of the
// linear-combination, blind-rotation and key-switching kernels over all of
// them.  Ciphertexts live in an arena of 2 KB slots; a wire is a slot plus a
// negation flag, so NOT, MOV and shifts by a constant cost nothing (§3: they
// need no bootstrapping).  Slots are reference counted: register bits,
// running instances and cached plans hold references.
//
// Fixed-shape work (one unit over a batch of n operand sets) is planned once
// — all descriptors of all levels uploaded, arena slots reserved — and
// replayed as a captured CUDA graph per (unit, shape).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ce_internal.h"
#include "ctx.h"
#include "launch.h"
#include "netlist.h"

namespace ce {

static_assert(sizeof(ce_trace_rec) == 8048, "trace record layout");

namespace {

constexpr uint32_t kSlotFalse = 0;  // the trivial ciphertext (0, -1/8)
constexpr uint32_t kSlotSink = 1;   // padding outputs land here
constexpr int kWidth = 16;          // register width
constexpr int kRegs = 8;

struct SRef {
  uint32_t slot = kSlotFalse;
  bool neg = false;
};

// Copy [n][n_in][501] packed ciphertexts into consecutive arena slots.
__global__ void copy_in_kernel(const uint32_t *__restrict__ in, uint32_t *__restrict__ arena,
                               uint32_t base) {
  const size_t c = blockIdx.x;
  for (int m = threadIdx.x; m < kLweWords; m += blockDim.x)
    arena[(size_t(base) + c) * kSlotWords + m] = in[c * kLweWords + m];
}

// out[c] = (neg ? -1 : 1) * arena[slot] for the (slot, neg) pairs in map.
__global__ void copy_out_kernel(const uint32_t *__restrict__ map, const uint32_t *__restrict__ arena,
                                uint32_t *__restrict__ out) {
  const size_t c = blockIdx.x;
  const uint32_t slot = map[2 * c], neg = map[2 * c + 1];
  for (int m = threadIdx.x; m < kLweWords; m += blockDim.x) {
    const uint32_t v = arena[size_t(slot) * kSlotWords + m];
    out[c * kLweWords + m] = neg ? 0u - v : v;
  }
}

// Gate trace: block r records sample r of a tick, the output at position
// floor(r * n_outs / samples) (padding outputs are skipped): the gate's
// operation, negation flags, client, its input slots' words and its output
// slot's words, copied after the tick's key switch on the same stream.
__global__ void trace_kernel(const GateJob *__restrict__ jobs, const GateOut *__restrict__ outs,
                             int n_outs, int samples, const uint32_t *__restrict__ arena,
                             ce_trace_rec *__restrict__ rec, unsigned long long *__restrict__ count,
                             unsigned long long cap, uint32_t tick) {
  const int k = int((long long)blockIdx.x * n_outs / samples);
  const GateOut o = outs[k];
  if (o.slot == kSlotSink) return;
  __shared__ unsigned long long idx;
  if (threadIdx.x == 0) idx = atomicAdd(count, 1ull);
  __syncthreads();
  if (idx >= cap) return;
  ce_trace_rec &R = rec[idx];
  const GateJob J1 = jobs[o.job1];
  const bool mux = o.job2 >= 0;
  const GateJob J2 = mux ? jobs[o.job2] : J1;
  if (threadIdx.x == 0) {
    R.op = mux ? 10 : J1.op;
    R.neg[0] = J1.neg_a;
    R.neg[1] = J1.neg_b;
    R.neg[2] = mux ? J2.neg_b : 0;
    R.client = int32_t(o.pad);
    R.tick = tick;
    R.index = uint32_t(k);
    R.pad = 0;
  }
  const uint32_t src[4] = {J1.a, J1.b, mux ? J2.b : kSlotFalse, o.slot};
  for (int m = threadIdx.x; m < 4 * kLweWords; m += blockDim.x) {
    const int w = m / kLweWords, j = m % kLweWords;
    const uint32_t v = (w == 2 && !mux) ? 0u : arena[size_t(src[w]) * kSlotWords + j];
    uint32_t *dst = w == 3 ? reinterpret_cast<uint32_t *>(&R.out)
                           : reinterpret_cast<uint32_t *>(&R.in[w]);
    dst[j] = v;
  }
}

// arena[dst] = (neg ? -1 : 1) * arena[src] for the (src, neg, dst) triples
// of map (register bits copied into and out of a program plan's slots).
__global__ void copy_slots_kernel(const uint32_t *__restrict__ map, uint32_t *__restrict__ arena) {
  const size_t c = blockIdx.x;
  const uint32_t src = map[3 * c], neg = map[3 * c + 1], dst = map[3 * c + 2];
  for (int m = threadIdx.x; m < kLweWords; m += blockDim.x) {
    const uint32_t v = arena[size_t(src) * kSlotWords + m];
    arena[size_t(dst) * kSlotWords + m] = neg ? 0u - v : v;
  }
}

__global__ void fill_false_kernel(uint32_t *__restrict__ arena) {
  for (int m = threadIdx.x; m < kSlotWords; m += blockDim.x)
    arena[m] = (m == kLweN) ? 0u - kMuEighth : 0u;
}

// Descriptors of one tick (one level of every participating instance).
struct TickDesc {
  std::vector<GateJob> jobs;
  std::vector<GateOut> outs;
  std::vector<const uint64_t *> grp_bsk;
  std::vector<const uint32_t *> tile_ksk;
  int G = 1, blocks = 1, tile = 1, jsplit = 1;
  const uint16_t *ks_planes = nullptr;  // single-client tick on the tensor-core key switch
  const uint16_t *br_hankel = nullptr;  // single-client tick on the tensor-core external product
};

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

struct Instance {
  const Netlist *net = nullptr;
  int client = 0;
  std::vector<SRef> wire;   // per netlist wire
  int level = 0;            // levels completed
  std::vector<SRef> result; // resolved outputs once complete
};

struct RegFile {
  SRef r[kRegs][kWidth];
  SRef nzcv[4];
};

struct Plan {
  int unit = 0, cond = 0, width = 0, client = 0, xp = 0, ks = 0;
  bool per_gate = false;             // planned for one launch per gate and step
  size_t n = 0;
  const uint32_t *d_in = nullptr;
  uint32_t *d_out = nullptr;
  uint32_t in_base = 0;
  std::vector<uint32_t> slots;       // all slots the plan owns
  uint8_t *d_desc = nullptr;         // descriptors of every level + output map
  struct Level {
    size_t jobs_off, outs_off, bsk_off, ksk_off;
    int n_jobs, n_outs, G, blocks, tile, jsplit;
    const uint16_t *ks_planes;
    const uint16_t *br_hankel;
  };
  std::vector<Level> levels;
  size_t map_off = 0;
  int n_in = 0, n_out = 0;
  size_t max_jobs = 0;
  cudaGraphExec_t exec = nullptr;
  uint64_t exec_gen = 0;  // scratch generation the graph was captured with
  int graph_launches = 0;
  uint64_t last_use = 0;
};

// A set of register programs (cleartext, no branches) planned once: every
// tick's descriptors recorded against slots the plan owns, then captured as
// one CUDA graph.  A run copies the clients' current register bits into the
// plan's input slots, replays the ticks, and copies the final register bits
// into fresh slots of the register files (copy maps uploaded per run).
constexpr int kRegBits = kRegs * kWidth + 4;  // 8 x 16 register bits + NZCV
struct ProgPlan {
  int xp = 0, ks = 0;                       // external-product form, key-switch engine
  bool per_gate = false;                    // one launch per gate and step
  bool fast_circuits = false;               // ADD / SUB / MUL on the low-latency circuits
  std::vector<int> clients;                 // per program
  std::vector<std::vector<uint8_t>> code;   // per program: instruction bytes
  std::vector<int> regfiles;                // distinct clients, in first-use order
  uint32_t in_base = 0;                     // kRegBits input slots per register file
  std::vector<uint32_t> slots;              // slots the plan owns (one reference each)
  std::vector<Plan::Level> levels;
  size_t max_jobs = 0;
  uint8_t *d_desc = nullptr;
  std::vector<std::vector<SRef>> final_refs;  // per register file: kRegBits refs
  size_t n_out_copies = 0;                  // final refs that are not constants
  uint32_t *d_map = nullptr;                // copy-in triples, then copy-out triples
  cudaGraphExec_t exec = nullptr;
  uint64_t exec_gen = 0;
  int graph_launches = 0;
  uint64_t last_use = 0;
  int ticks = 0;
};

class Engine {
 public:
  explicit Engine(ce_ctx *c) : ctx(c) {}
  ~Engine() {
    for (auto &p : plans) drop_plan(*p);
    for (auto &p : pplans) drop_prog_plan(*p);
    for (int i = 0; i < 2; ++i) {
      if (h_desc[i]) cudaFreeHost(h_desc[i]);
      dev_free(d_desc[i]);
      if (desc_ev[i]) cudaEventDestroy(desc_ev[i]);
    }
    dev_free(arena);
    dev_free(trace_rec);
    dev_free(trace_count);
    dev_free(io_in);
    dev_free(io_out);
    if (cap_stream) cudaStreamDestroy(cap_stream);
  }

  ce_status init() {
    ce_status s = reserve(1 << 14);
    if (s != CE_OK) return s;
    rc.assign(2, 1);  // FALSE and sink are permanent
    next_slot = 2;
    fill_false_kernel<<<1, 512, 0, ctx->stream>>>(arena);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&desc_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_error(e, "engine init");
    return CE_OK;
  }

  // ------------------------------------------------------------ arena ---
  ce_status reserve(size_t slots) {
    if (slots <= cap) return CE_OK;
    size_t ncap = cap ? cap : 1;
    while (ncap < slots) ncap *= 2;
    uint32_t *na = nullptr;
    cudaError_t e = dev_malloc(&na, ncap * kSlotWords * sizeof(uint32_t));
    if (e != cudaSuccess) return set_error(CE_ENOMEM, "engine: arena allocation failed");
    if (arena) {
      // rare: wait for all work that may touch the old arena, then move it
      e = cudaDeviceSynchronize();
      if (e == cudaSuccess)
        e = cudaMemcpy(na, arena, cap * kSlotWords * sizeof(uint32_t), cudaMemcpyDeviceToDevice);
      dev_free(arena);
      // plans captured the old address
      for (auto &p : plans) drop_graph(*p);
      for (auto &p : pplans) drop_prog_graph(*p);
    }
    arena = na;
    cap = ncap;
    return e == cudaSuccess ? CE_OK : cuda_error(e, "engine: arena growth");
  }
  ce_status alloc(uint32_t *out) {
    if (!free_.empty()) {
      *out = free_.back();
      free_.pop_back();
      rc[*out] = 1;
      return CE_OK;
    }
    if (next_slot >= cap) {
      ce_status s = reserve(next_slot + 1);
      if (s != CE_OK) return s;
    }
    *out = next_slot++;
    if (rc.size() <= *out) rc.resize(*out + 1, 0);
    rc[*out] = 1;
    return CE_OK;
  }
  void ref(const SRef &r) {
    if (r.slot > kSlotSink) ++rc[r.slot];
  }
  void unref(const SRef &r) {
    if (r.slot > kSlotSink && --rc[r.slot] == 0) free_.push_back(r.slot);
  }

  const Netlist *netlist(int unit, int cond, int width = kWidth) {
    const int key = (width * 64 + unit) * 16 + cond;
    auto it = nets.find(key);
    if (it != nets.end()) return &it->second;
    Netlist n;
    if (!build_unit(unit, width, unit == kUnitCsel ? cond : 0, &n)) return nullptr;
    return &nets.emplace(key, std::move(n)).first->second;
  }

  RegFile &regs(int client) {
    auto it = rf.find(client);
    if (it == rf.end()) it = rf.emplace(client, RegFile{}).first;
    return it->second;
  }
  void drop_client(int client) {
    auto it = rf.find(client);
    if (it == rf.end()) return;
    for (auto &r : it->second.r)
      for (auto &b : r) unref(b);
    for (auto &b : it->second.nzcv) unref(b);
    rf.erase(it);
    for (auto pit = plans.begin(); pit != plans.end();) {
      if ((*pit)->client == client) {
        drop_plan(**pit);
        pit = plans.erase(pit);
      } else {
        ++pit;
      }
    }
    for (auto pit = pplans.begin(); pit != pplans.end();) {
      const auto &cl = (*pit)->regfiles;
      if (std::find(cl.begin(), cl.end(), client) != cl.end()) {
        drop_prog_plan(**pit);
        pit = pplans.erase(pit);
      } else {
        ++pit;
      }
    }
  }

  // ---------------------------------------------------------- instance ---
  ce_status start(Instance &in, const Netlist *net, int client, const std::vector<SRef> &inputs) {
    in.net = net;
    in.client = client;
    in.level = 0;
    in.wire.assign(net->n_wires, SRef{});
    for (int i = 0; i < net->n_inputs; ++i) {
      in.wire[i] = inputs[i];
      ref(inputs[i]);
    }
    return CE_OK;
  }
  SRef resolve(const Instance &in, const Ref &r) const {
    if (r.wire < 0) return SRef{kSlotFalse, r.neg};
    const SRef &w = in.wire[r.wire];
    return SRef{w.slot, w.neg != r.neg};
  }
  // Outputs taken (one reference each), then the instance's own released.
  void complete(Instance &in) {
    in.result.clear();
    for (const Ref &r : in.net->outputs) {
      const SRef s = resolve(in, r);
      ref(s);
      in.result.push_back(s);
    }
    for (const SRef &w : in.wire) unref(w);
    in.wire.clear();
  }

  // Builds the descriptors of the next level of every instance (grouped by
  // client; groups of G jobs and tiles of `tile` outputs never mix clients).
  ce_status build_tick(const std::vector<Instance *> &act, TickDesc &t) {
    std::vector<Instance *> order(act);
    std::stable_sort(order.begin(), order.end(),
                     [](const Instance *a, const Instance *b) { return a->client < b->client; });
    size_t total_jobs = 0, total_outs = 0;
    for (Instance *in : order) {
      const Netlist &n = *in->net;
      for (int g = n.level_begin[in->level]; g < n.level_begin[in->level + 1]; ++g) {
        total_jobs += n.gates[g].op == kOpMux ? 2 : 1;
        ++total_outs;
      }
    }
    br_shape(ctx, total_jobs, &t.G, &t.blocks);
    ks_shape(ctx, total_outs, &t.tile, &t.jsplit);
    if (ctx->per_gate) {  // one key per job and per output: launches of one gate each
      t.G = 3;
      t.tile = 1;
      t.jsplit = 1;
    }
    t.jobs.clear();
    t.outs.clear();
    t.grp_bsk.clear();
    t.tile_ksk.clear();
    size_t i = 0;
    while (i < order.size()) {
      const int client = order[i]->client;
      const Client &cl = ctx->clients[client];
      const size_t job0 = t.jobs.size(), out0 = t.outs.size();
      for (; i < order.size() && order[i]->client == client; ++i) {
        Instance &in = *order[i];
        const Netlist &n = *in.net;
        for (int g = n.level_begin[in.level]; g < n.level_begin[in.level + 1]; ++g) {
          const NGate &x = n.gates[g];
          uint32_t slot;
          ce_status s = alloc(&slot);
          if (s != CE_OK) return s;
          in.wire[x.out] = SRef{slot, false};
          const SRef a = resolve(in, x.a), b = resolve(in, x.b);
          GateOut o{};
          o.slot = slot;
          o.pad = uint32_t(client);  // read by the gate trace
          o.job1 = int32_t(t.jobs.size());
          if (x.op == kOpMux) {
            const SRef c = resolve(in, x.c);
            t.jobs.push_back(GateJob{a.slot, b.slot, 10, a.neg, b.neg, 0});
            t.jobs.push_back(GateJob{a.slot, c.slot, 11, a.neg, c.neg, 0});
            o.job2 = o.job1 + 1;
          } else {
            t.jobs.push_back(GateJob{a.slot, b.slot, x.op, a.neg, b.neg, 0});
            o.job2 = -1;
          }
          t.outs.push_back(o);
        }
      }
      const int gsz = t.G == 3 ? 1 : t.G;  // jobs per key group of the launch shape
      while ((t.jobs.size() - job0) % gsz) t.jobs.push_back(GateJob{kSlotFalse, kSlotFalse, 0, 0, 0, 0});
      for (size_t g = job0; g < t.jobs.size(); g += gsz) t.grp_bsk.push_back(cl.bsk);
      while ((t.outs.size() - out0) % t.tile) t.outs.push_back(GateOut{int32_t(job0), -1, kSlotSink, 0});
      for (size_t o = out0; o < t.outs.size(); o += t.tile) t.tile_ksk.push_back(cl.ksk);
    }
    // one client: the key switch may run on the tensor cores with its planes,
    // and the external products too (Toeplitz form) when selected
    t.ks_planes = nullptr;
    t.br_hankel = nullptr;
    const bool one_client = !order.empty() && order.front()->client == order.back()->client;
    if (one_client && !ctx->per_gate && ks_use_tensor(ctx, total_outs))
      t.ks_planes = ctx->clients[order.front()->client].ksk_planes;
    if (one_client && !ctx->per_gate && ctx->cfg_xp == 1) {
      Client &cl = ctx->clients[order.front()->client];
      ce_status hs = ensure_hankel(ctx, &cl);
      if (hs != CE_OK) return hs;
      t.br_hankel = cl.bsk_hankel;
    }
    // the padded batch may need more blocks than the unpadded estimate
    const size_t groups = t.jobs.size() / (t.G == 3 ? 1 : t.G);
    t.blocks = int(std::min<size_t>(groups, size_t(ctx->sms) * (t.G == 1 ? 2 : 1)));
    if (ctx->per_gate) t.blocks = 1;
    return CE_OK;
  }

  // Stages descriptors in pinned memory and copies them to the device.
  ce_status stage(const TickDesc &t, cudaStream_t st, uint8_t **dev, size_t *offs) {
    size_t off = 0;
    offs[0] = off;
    off = align16(off + t.jobs.size() * sizeof(GateJob));
    offs[1] = off;
    off = align16(off + t.outs.size() * sizeof(GateOut));
    offs[2] = off;
    off = align16(off + t.grp_bsk.size() * sizeof(void *));
    offs[3] = off;
    off = align16(off + t.tile_ksk.size() * sizeof(void *));
    const int b = desc_i;
    desc_i ^= 1;
    cudaError_t e = cudaEventSynchronize(desc_ev[b]);  // previous use of this buffer copied
    if (e != cudaSuccess) return cuda_error(e, "engine stage");
    if (off > desc_cap[b]) {
      if (h_desc[b]) cudaFreeHost(h_desc[b]);
      dev_free(d_desc[b]);
      h_desc[b] = nullptr;
      d_desc[b] = nullptr;
      size_t c = std::max<size_t>(off, 1 << 16) * 2;
      e = cudaMallocHost(&h_desc[b], c);
      if (e == cudaSuccess) e = dev_malloc(&d_desc[b], c);
      if (e != cudaSuccess) {
        desc_cap[b] = 0;
        return set_error(CE_ENOMEM, "engine: descriptor buffers");
      }
      desc_cap[b] = c;
    }
    std::memcpy(h_desc[b] + offs[0], t.jobs.data(), t.jobs.size() * sizeof(GateJob));
    std::memcpy(h_desc[b] + offs[1], t.outs.data(), t.outs.size() * sizeof(GateOut));
    std::memcpy(h_desc[b] + offs[2], t.grp_bsk.data(), t.grp_bsk.size() * sizeof(void *));
    std::memcpy(h_desc[b] + offs[3], t.tile_ksk.data(), t.tile_ksk.size() * sizeof(void *));
    e = cudaMemcpyAsync(d_desc[b], h_desc[b], off, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(desc_ev[b], st);
    if (e != cudaSuccess) return cuda_error(e, "engine stage copy");
    *dev = d_desc[b];
    return CE_OK;
  }

  // Comparison mode (ce_set_level_batching off): every gate's steps as
  // launches of their own — one job's gather + linear combination, one job's
  // blind rotation (one gate, latency shape), one output's extraction + key
  // switch — in place of the level's batched launches.  The tick was planned
  // with one key per job and per output.
  ce_status launch_level_per_gate(const GateJob *jobs, int n_jobs, const GateOut *outs,
                                  int n_outs, const uint64_t *const *grp_bsk,
                                  const uint32_t *const *tile_ksk, cudaStream_t st,
                                  int *launches) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n_jobs && e == cudaSuccess; ++k) {
      uint16_t *abar = ctx->abar + size_t(k) * kAbarStride;
      e = timed(ctx, 0, st, [&] {
        return launch_lincomb_gather(jobs + k, arena, abar, 1, ctx->err, st);
      });
      if (e == cudaSuccess)
        e = timed(ctx, 1, st, [&] {
          return launch_blind_rotate(nullptr, abar, ctx->acc + size_t(k) * 2 * kRingN, 1, ctx->tw,
                                     ctx->err, 3, 1, st, grp_bsk + k);
        });
      *launches += 2;
    }
    for (int o = 0; o < n_outs && e == cudaSuccess; ++o) {
      e = timed(ctx, 2, st, [&] {
        return launch_extract_keyswitch_ex(ctx->acc, nullptr, tile_ksk + o, outs + o, arena, 1, 2,
                                           1, 1, st);
      });
      ++*launches;
    }
    if (e != cudaSuccess) return cuda_error(e, "engine per-gate launch");
    if (trace_per_tick > 0) {
      const int samples = std::min(trace_per_tick, n_outs);
      trace_kernel<<<unsigned(samples), 256, 0, st>>>(jobs, outs, n_outs, samples, arena, trace_rec,
                                                       trace_count, trace_cap, trace_tick++);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "gate trace");
      ++*launches;
    }
    return CE_OK;
  }

  // Launches one level: gather + linear combination, blind rotation, key
  // switching into the arena.
  ce_status launch_level(const GateJob *jobs, int n_jobs, const GateOut *outs, int n_outs,
                         const uint64_t *const *grp_bsk, const uint32_t *const *tile_ksk, int G,
                         int blocks, int tile, int jsplit, const uint16_t *ks_planes,
                         const uint16_t *br_hankel, cudaStream_t st, int *launches) {
    ce_status s = ensure_job_scratch(ctx, n_jobs);
    if (s != CE_OK) return s;
    if (ctx->per_gate) return launch_level_per_gate(jobs, n_jobs, outs, n_outs, grp_bsk, tile_ksk,
                                                    st, launches);
    cudaError_t e = timed(ctx, 0, st, [&] {
      return launch_lincomb_gather(jobs, arena, ctx->abar, n_jobs, ctx->err, st);
    });
    if (e == cudaSuccess && br_hankel) {
      const int ctas = blind_rotate_tc_ctas(ctx->sms, n_jobs);
      int tc_launches = 0;
      e = timed(ctx, 1, st, [&] {
        return launch_blind_rotate_tc(br_hankel, ctx->abar, ctx->acc, n_jobs, ctx->tt_digits,
                                      ctas, ctx->err, st, &tc_launches, mma_events(ctx));
      });
      keep_mma_events(ctx);
      *launches += tc_launches - 1;  // one blind-rotation launch is counted below
    } else if (e == cudaSuccess) {
      int br_launches = 0;
      e = timed(ctx, 1, st, [&] {
        return launch_blind_rotate(nullptr, ctx->abar, ctx->acc, n_jobs, ctx->tw, ctx->err, G,
                                   blocks, st, grp_bsk, &br_launches);
      });
      *launches += br_launches - 1;  // one blind-rotation launch is counted below
    }
    int split = jsplit;
    if (ks_planes) {
      int n_tile, out_tiles;
      keyswitch_tc_shape(ctx->sms, n_outs, &n_tile, &out_tiles, &split);
      if (e == cudaSuccess && split > 1) e = launch_zero_slots(outs, arena, n_outs, st);
      if (e == cudaSuccess)
        e = timed(ctx, 2, st, [&] {
          return launch_keyswitch_tc(ctx->acc, ks_planes, outs, arena, n_outs, 2, n_tile,
                                     out_tiles, split, ctx->ksh, ksh_ld(ctx->job_cap), ctx->err,
                                     st);
        });
      ++*launches;  // the rounding pass
    } else {
      if (e == cudaSuccess && jsplit > 1) e = launch_zero_slots(outs, arena, n_outs, st);
      if (e == cudaSuccess)
        e = timed(ctx, 2, st, [&] {
          return launch_extract_keyswitch_ex(ctx->acc, nullptr, tile_ksk, outs, arena, n_outs, 2,
                                             tile, jsplit, st);
        });
    }
    if (e != cudaSuccess) return cuda_error(e, "engine level launch");
    *launches += 3 + (split > 1 ? 1 : 0);
    if (trace_per_tick > 0) {
      const int samples = std::min(trace_per_tick, n_outs);
      trace_kernel<<<unsigned(samples), 256, 0, st>>>(jobs, outs, n_outs, samples, arena, trace_rec,
                                                       trace_count, trace_cap, trace_tick++);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_error(e, "gate trace");
      ++*launches;
    }
    return CE_OK;
  }

  ce_status tick(std::vector<Instance *> &act, cudaStream_t st, int *launches) {
    TickDesc t;
    ce_status s = build_tick(act, t);
    if (s != CE_OK) return s;
    uint8_t *dev;
    size_t offs[4];
    s = stage(t, st, &dev, offs);
    if (s != CE_OK) return s;
    s = launch_level(reinterpret_cast<const GateJob *>(dev + offs[0]), int(t.jobs.size()),
                     reinterpret_cast<const GateOut *>(dev + offs[1]), int(t.outs.size()),
                     reinterpret_cast<const uint64_t *const *>(dev + offs[2]),
                     reinterpret_cast<const uint32_t *const *>(dev + offs[3]), t.G, t.blocks,
                     t.tile, t.jsplit, t.ks_planes, t.br_hankel, st, launches);
    if (s != CE_OK) return s;
    for (Instance *in : act) ++in->level;
    return CE_OK;
  }

  // ------------------------------------------------------------- plans ---
  void drop_graph(Plan &p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    p.exec = nullptr;
  }
  void drop_plan(Plan &p) {
    drop_graph(p);
    dev_free(p.d_desc);
    p.d_desc = nullptr;
    for (uint32_t sl : p.slots) unref(SRef{sl, false});
    p.slots.clear();
  }
  void drop_prog_graph(ProgPlan &p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    p.exec = nullptr;
  }
  void drop_prog_plan(ProgPlan &p) {
    drop_prog_graph(p);
    dev_free(p.d_desc);
    dev_free(p.d_map);
    p.d_desc = nullptr;
    p.d_map = nullptr;
    for (auto &refs : p.final_refs)
      for (const SRef &r : refs) unref(r);
    p.final_refs.clear();
    for (uint32_t sl : p.slots) unref(SRef{sl, false});
    p.slots.clear();
  }
  // Appends a built tick's descriptors to a plan blob; the plan takes a
  // reference on every slot the tick writes, so no later work reuses it.
  Plan::Level record_level(const TickDesc &t, std::vector<uint8_t> &blob,
                           std::vector<uint32_t> &owned) {
    auto put = [&](const void *src, size_t bytes) {
      const size_t off = align16(blob.size());
      blob.resize(off + bytes);
      if (bytes) std::memcpy(blob.data() + off, src, bytes);
      return off;
    };
    Plan::Level lv{};
    lv.n_jobs = int(t.jobs.size());
    lv.n_outs = int(t.outs.size());
    lv.G = t.G;
    lv.blocks = t.blocks;
    lv.tile = t.tile;
    lv.jsplit = t.jsplit;
    lv.ks_planes = t.ks_planes;
    lv.br_hankel = t.br_hankel;
    lv.jobs_off = put(t.jobs.data(), t.jobs.size() * sizeof(GateJob));
    lv.outs_off = put(t.outs.data(), t.outs.size() * sizeof(GateOut));
    lv.bsk_off = put(t.grp_bsk.data(), t.grp_bsk.size() * sizeof(void *));
    lv.ksk_off = put(t.tile_ksk.data(), t.tile_ksk.size() * sizeof(void *));
    for (const GateOut &o : t.outs)
      if (o.slot > kSlotSink) {
        ref(SRef{o.slot, false});
        owned.push_back(o.slot);
      }
    return lv;
  }
  // Launches recorded levels whose descriptors live at d_desc.
  ce_status launch_levels(const std::vector<Plan::Level> &levels, const uint8_t *d_desc,
                          cudaStream_t st, int *launches) {
    for (const Plan::Level &lv : levels) {
      ce_status s = launch_level(reinterpret_cast<const GateJob *>(d_desc + lv.jobs_off), lv.n_jobs,
                                 reinterpret_cast<const GateOut *>(d_desc + lv.outs_off), lv.n_outs,
                                 reinterpret_cast<const uint64_t *const *>(d_desc + lv.bsk_off),
                                 reinterpret_cast<const uint32_t *const *>(d_desc + lv.ksk_off),
                                 lv.G, lv.blocks, lv.tile, lv.jsplit, lv.ks_planes, lv.br_hankel, st,
                                 launches);
      if (s != CE_OK) return s;
    }
    return CE_OK;
  }

  ce_status make_plan(int unit, int cond, int width, int client, size_t n, const uint32_t *d_in,
                      uint32_t *d_out, Plan **out) {
    for (auto &p : plans)
      if (p->unit == unit && p->cond == cond && p->width == width && p->client == client &&
          p->n == n && p->d_in == d_in && p->d_out == d_out && p->xp == ctx->cfg_xp &&
          p->ks == ctx->cfg_ks && p->per_gate == ctx->per_gate) {
        p->last_use = ++use_clock;
        *out = p.get();
        return CE_OK;
      }
    const Netlist *net = netlist(unit, cond, width);
    if (!net) return set_error(CE_EINVAL, "engine: bad unit or width");
    if (plans.size() >= 8) {  // evict the least recently used plan
      auto lru = std::min_element(plans.begin(), plans.end(), [](const auto &a, const auto &b) {
        return a->last_use < b->last_use;
      });
      drop_plan(**lru);
      plans.erase(lru);
    }
    auto p = std::make_unique<Plan>();
    p->unit = unit;
    p->cond = cond;
    p->width = width;
    p->client = client;
    p->xp = ctx->cfg_xp;
    p->ks = ctx->cfg_ks;
    p->per_gate = ctx->per_gate;
    p->n = n;
    p->d_in = d_in;
    p->d_out = d_out;
    p->n_in = net->n_inputs;
    p->n_out = int(net->outputs.size());
    // input slots: one consecutive block, so copy-in needs no map
    const size_t n_in_slots = n * p->n_in;
    ce_status s = reserve(next_slot + n_in_slots + 1);
    if (s != CE_OK) return s;
    p->in_base = uint32_t(next_slot);
    for (size_t k = 0; k < n_in_slots; ++k) {
      const uint32_t sl = uint32_t(next_slot++);
      if (rc.size() <= sl) rc.resize(sl + 1, 0);
      rc[sl] = 1;  // owned by the plan
      p->slots.push_back(sl);
    }
    std::vector<Instance> inst(n);
    for (size_t i = 0; i < n; ++i) {
      std::vector<SRef> in(p->n_in);
      for (int k = 0; k < p->n_in; ++k) in[k] = SRef{uint32_t(p->in_base + i * p->n_in + k), false};
      start(inst[i], net, client, in);
    }
    std::vector<Instance *> act;
    for (auto &x : inst) act.push_back(&x);
    // descriptors of every level, appended to one blob
    std::vector<uint8_t> blob;
    auto put = [&](const void *src, size_t bytes) {
      const size_t off = align16(blob.size());
      blob.resize(off + bytes);
      if (bytes) std::memcpy(blob.data() + off, src, bytes);
      return off;
    };
    for (int L = 0; L < net->depth; ++L) {
      TickDesc t;
      s = build_tick(act, t);
      if (s != CE_OK) return s;
      for (Instance *in : act) ++in->level;
      p->max_jobs = std::max(p->max_jobs, t.jobs.size());
      // the plan keeps every slot its levels write (taken before the
      // instances release theirs below)
      p->levels.push_back(record_level(t, blob, p->slots));
    }
    std::vector<uint32_t> map;
    for (auto &x : inst) {
      complete(x);
      for (const SRef &r : x.result) {
        map.push_back(r.slot);
        map.push_back(r.neg ? 1u : 0u);
        if (r.slot > kSlotSink) p->slots.push_back(r.slot);  // reference taken by complete()
      }
    }
    p->map_off = put(map.data(), map.size() * sizeof(uint32_t));
    cudaError_t e = dev_malloc(&p->d_desc, blob.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_desc, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_error(e, "engine plan upload");
    p->last_use = ++use_clock;
    *out = p.get();
    plans.push_back(std::move(p));
    return CE_OK;
  }

  ce_status run_plan(Plan &p, cudaStream_t st, int *launches) {
    ce_status s = ensure_job_scratch(ctx, p.max_jobs);
    if (s != CE_OK) return s;
    copy_in_kernel<<<unsigned(p.n * p.n_in), 128, 0, st>>>(p.d_in, arena, p.in_base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "copy_in");
    ++*launches;
    s = launch_levels(p.levels, p.d_desc, st, launches);
    if (s != CE_OK) return s;
    copy_out_kernel<<<unsigned(p.n * p.n_out), 128, 0, st>>>(
        reinterpret_cast<const uint32_t *>(p.d_desc + p.map_off), arena, p.d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "copy_out");
    ++*launches;
    return CE_OK;
  }

  ce_status eval_unit(int unit, int cond, int width, int client, const uint32_t *d_in,
                      uint32_t *d_out,
                      size_t n, cudaStream_t st, int *launches) {
    Plan *p;
    ce_status s = make_plan(unit, cond, width, client, n, d_in, d_out, &p);
    if (s != CE_OK) return s;
    if (!use_graphs || ctx->profile || trace_per_tick > 0) return run_plan(*p, st, launches);
    s = ensure_job_scratch(ctx, p->max_jobs);
    if (s != CE_OK) return s;
    if (p->exec && p->exec_gen != ctx->scratch_gen) drop_graph(*p);  // scratch was replaced
    if (!p->exec) {
      // capture once on the engine's own stream, then replay on any stream
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return cuda_error(e, "begin capture");
      int dummy = 0;
      s = run_plan(*p, cap_stream, &dummy);
      e = cudaStreamEndCapture(cap_stream, &g);
      if (s != CE_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_error(e, "graph instantiate");
      p->graph_launches = dummy;
      p->exec_gen = ctx->scratch_gen;
    }
    cudaError_t e = cudaGraphLaunch(p->exec, st);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
    *launches += p->graph_launches;
    return CE_OK;
  }

  ce_ctx *ctx;
  uint32_t *arena = nullptr;
  size_t cap = 0, next_slot = 0;
  std::vector<uint32_t> rc, free_;
  std::map<int, Netlist> nets;
  std::map<int, RegFile> rf;
  uint8_t *h_desc[2] = {nullptr, nullptr}, *d_desc[2] = {nullptr, nullptr};
  size_t desc_cap[2] = {0, 0};
  cudaEvent_t desc_ev[2] = {nullptr, nullptr};
  int desc_i = 0;
  std::list<std::unique_ptr<Plan>> plans;
  std::list<std::unique_ptr<ProgPlan>> pplans;
  uint64_t use_clock = 0;
  bool use_graphs = true;
  cudaStream_t cap_stream = nullptr;
  // staging buffers of ce_unit_eval (host-buffer calls), grown on demand
  uint32_t *io_in = nullptr, *io_out = nullptr;
  size_t io_in_cap = 0, io_out_cap = 0;
  ce_status ensure_unit_io(size_t in_bytes, size_t out_bytes) {
    if (in_bytes > io_in_cap) {
      dev_free(io_in);
      io_in = nullptr;
      io_in_cap = 0;
      if (dev_malloc(&io_in, in_bytes) != cudaSuccess)
        return set_error(CE_ENOMEM, "ce_unit_eval: staging allocation failed");
      io_in_cap = in_bytes;
    }
    if (out_bytes > io_out_cap) {
      dev_free(io_out);
      io_out = nullptr;
      io_out_cap = 0;
      if (dev_malloc(&io_out, out_bytes) != cudaSuccess)
        return set_error(CE_ENOMEM, "ce_unit_eval: staging allocation failed");
      io_out_cap = out_bytes;
    }
    return CE_OK;
  }
  // gate trace (ce_trace_enable): records of sampled gates of every tick
  int trace_per_tick = 0;
  ce_trace_rec *trace_rec = nullptr;
  unsigned long long *trace_count = nullptr;
  unsigned long long trace_cap = 0;
  uint32_t trace_tick = 0;
  // one host thread at a time inside the engine (a serving thread and
  // register reads of other threads may meet here)
  std::recursive_mutex mu;
};

void serve_runs_forget(Engine *e);
void engine_destroy(Engine *e) {
  if (!e) return;
  serve_runs_forget(e);
  delete e;
}
void engine_drop_client(Engine *e, int client) {
  if (!e) return;
  std::lock_guard<std::recursive_mutex> lock(e->mu);
  e->drop_client(client);
}

namespace {

ce_status get_engine(ce_ctx *ctx, Engine **out) {
  if (!ctx->engine) {
    Engine *e = new Engine(ctx);
    ce_status s = e->init();
    if (s != CE_OK) {
      delete e;
      return s;
    }
    ctx->engine = e;
  }
  *out = ctx->engine;
  return CE_OK;
}

bool live_client(ce_ctx *ctx, int client) {
  return client >= 0 && client < int(ctx->clients.size()) && ctx->clients[client].live;
}

// Instruction set (16-bit registers R0..R7, encrypted NZCV).
enum Opcode : uint8_t {
  kAdd = 0, kSub = 1, kAnd = 2, kOrr = 3, kLsl = 4, kLslImm = 5, kMul = 6, kUdiv = 7,
  kCmp = 8, kCsel = 9, kMov = 10, kMovImm = 11, kLsr = 12, kAsr = 13, kLsrImm = 14,
  kAsrImm = 15, kEor = 16, kOrn = 17, kMvn = 18, kAndImm = 19, kOrrImm = 20, kEorImm = 21,
  kBfc = 22, kBfi = 23, kRbit = 24, kRev = 25, kAdds = 26, kSubs = 27, kSmulh = 28,
  kUmulh = 29, kBcond = 30, kB = 31, kOpcodes = 32
};

// Instructions that only move, negate or fix wires (no bootstrap, §5 "Data
// movement": TFHE's COPY/NOT/CONSTANT): the new value of bit j of rd.
// Returns false for an instruction that needs gates.
bool wire_move(const ce_insn &I, const SRef *rd, const SRef *rn, int j, SRef *out) {
  const int sh = I.imm % kWidth;
  const SRef fls{kSlotFalse, false}, tru{kSlotFalse, true};
  const bool ib = (I.imm >> j) & 1;  // immediate bit (8-bit immediates: zero above bit 7)
  const int lsb = I.imm & 15, width = (I.imm >> 4) + 1;  // BFC/BFI field
  const bool in_field = j >= lsb && j < lsb + width;
  switch (I.op) {
    case kMov: *out = rn[j]; return true;
    case kMovImm: *out = ib ? tru : fls; return true;
    case kLslImm: *out = j >= sh ? rn[j - sh] : fls; return true;
    case kLsrImm: *out = j + sh < kWidth ? rn[j + sh] : fls; return true;
    case kAsrImm: *out = j + sh < kWidth ? rn[j + sh] : rn[kWidth - 1]; return true;
    case kMvn: *out = SRef{rn[j].slot, !rn[j].neg}; return true;
    case kAndImm: *out = ib ? rn[j] : fls; return true;
    case kOrrImm: *out = ib ? tru : rn[j]; return true;
    case kEorImm: *out = ib ? SRef{rn[j].slot, !rn[j].neg} : rn[j]; return true;
    case kBfc: *out = in_field ? fls : rd[j]; return true;
    case kBfi: *out = in_field ? rn[j - lsb] : rd[j]; return true;
    case kRbit: *out = rn[kWidth - 1 - j]; return true;
    case kRev: *out = rn[j ^ 8]; return true;  // byte swap of a 16-bit register
    default: return false;
  }
}

// The unit an instruction runs; with low-latency circuits selected, ADD, SUB,
// MUL and UDIV run the same operations on the MUX-carry adders and the tree
// multiplier (fewer levels).
int unit_of(uint8_t op, bool low_latency) {
  if (low_latency) {
    if (op == kAdd) return kUnitAddMux;
    if (op == kSub) return kUnitSubMux;
    if (op == kMul) return kUnitMulTree;
    if (op == kUdiv) return kUnitUdivMux;
  }
  switch (op) {
    case kAdd: return kUnitAdd;
    case kSub: return kUnitSub;
    case kAnd: return kUnitAnd;
    case kOrr: return kUnitOrr;
    case kLsl: return kUnitLsl;
    case kMul: return kUnitMul;
    case kUdiv: return kUnitUdiv;
    case kCmp: return kUnitCmp;
    case kCsel: return kUnitCsel;
    case kLsr: return kUnitLsr;
    case kAsr: return kUnitAsr;
    case kEor: return kUnitEor;
    case kOrn: return kUnitOrn;
    case kAdds: return kUnitAdds;
    case kSubs: return kUnitSubs;
    case kSmulh: return kUnitSmull;
    case kUmulh: return kUnitUmull;
    default: return -1;
  }
}

struct Run {
  int client = 0;
  const ce_insn *code = nullptr;
  size_t n = 0, pc = 0;
  std::unique_ptr<Instance> cur;
  ce_insn one{};           // storage for single-instruction runs (serving)
  RegFile *rf = nullptr;   // register file to use instead of the client's (planning)
};

// In-flight single instructions of the serving loop, by client.
std::map<Engine *, std::map<int, Run>> g_serve_runs;

// Executes free instructions until one needs gates (started as an instance)
// or the program ends.
ce_status advance(Engine &E, Run &r) {
  RegFile &R = r.rf ? *r.rf : E.regs(r.client);
  while (!r.cur && r.pc < r.n) {
    const ce_insn &I = r.code[r.pc];
    if (I.op >= kOpcodes || I.rd >= kRegs || I.rn >= kRegs || I.rm >= kRegs || I.cond > 13)
      return set_error(CE_EINVAL, "ce_exec: malformed instruction at index " + std::to_string(r.pc));
    if (I.op == kBcond || I.op == kB)
      return set_error(CE_EINVAL, "ce_exec: branch at index " + std::to_string(r.pc) +
                                      " (programs with branches run through ce_exec_branching)");
    SRef probe;
    if (wire_move(I, R.r[I.rd], R.r[I.rn], 0, &probe)) {
      SRef nv[kWidth];
      for (int j = 0; j < kWidth; ++j) {
        wire_move(I, R.r[I.rd], R.r[I.rn], j, &nv[j]);
        E.ref(nv[j]);
      }
      for (int j = 0; j < kWidth; ++j) {
        E.unref(R.r[I.rd][j]);
        R.r[I.rd][j] = nv[j];
      }
      ++r.pc;
      continue;
    }
    const Netlist *net = E.netlist(unit_of(I.op, E.ctx->fast_circuits), I.cond);
    std::vector<SRef> in;
    for (int j = 0; j < kWidth; ++j) in.push_back(R.r[I.rn][j]);
    for (int j = 0; j < kWidth; ++j) in.push_back(R.r[I.rm][j]);
    if (I.op == kCsel)
      for (int k = 0; k < 4; ++k) in.push_back(R.nzcv[k]);
    r.cur.reset(new Instance());
    E.start(*r.cur, net, r.client, in);
  }
  return CE_OK;
}

void retire(Engine &E, Run &r) {
  const ce_insn &I = r.code[r.pc];
  E.complete(*r.cur);
  RegFile &R = r.rf ? *r.rf : E.regs(r.client);
  // CMP: result = NZCV; ADDS/SUBS: rd bits then NZCV; SMULH/UMULH: the
  // high half of the 32-bit product; others: rd bits
  const bool flags = I.op == kCmp || I.op == kAdds || I.op == kSubs;
  const int first_flag = I.op == kCmp ? 0 : kWidth;
  const int first_bit = (I.op == kSmulh || I.op == kUmulh) ? kWidth : 0;
  if (I.op != kCmp)
    for (int j = 0; j < kWidth; ++j) {
      E.unref(R.r[I.rd][j]);
      R.r[I.rd][j] = r.cur->result[first_bit + j];
    }
  if (flags)
    for (int k = 0; k < 4; ++k) {
      E.unref(R.nzcv[k]);
      R.nzcv[k] = r.cur->result[first_flag + k];
    }
  r.cur.reset();
  ++r.pc;
}

// ------------------------------------------------------- program plans ---
bool plan_matches(const ce_ctx *ctx, const ProgPlan &p, size_t n_prog, const int *clients,
                  const ce_insn *const *progs, const size_t *lens) {
  if (p.clients.size() != n_prog || p.xp != ctx->cfg_xp || p.ks != ctx->cfg_ks ||
      p.per_gate != ctx->per_gate || p.fast_circuits != ctx->fast_circuits)
    return false;
  for (size_t i = 0; i < n_prog; ++i) {
    if (p.clients[i] != clients[i] || p.code[i].size() != lens[i] * sizeof(ce_insn)) return false;
    if (lens[i] && std::memcmp(p.code[i].data(), progs[i], lens[i] * sizeof(ce_insn)) != 0)
      return false;
  }
  return true;
}

// Plans a program set: runs the tick loop of exec_programs on the host
// against plan-owned input slots, recording every tick's descriptors.
// Malformed programs fail here, before anything is enqueued.
ce_status make_prog_plan(Engine &E, size_t n_prog, const int *clients, const ce_insn *const *progs,
                         const size_t *lens, ProgPlan **out) {
  auto p = std::make_unique<ProgPlan>();
  p->xp = E.ctx->cfg_xp;
  p->ks = E.ctx->cfg_ks;
  p->per_gate = E.ctx->per_gate;
  p->fast_circuits = E.ctx->fast_circuits;
  for (size_t i = 0; i < n_prog; ++i) {
    p->clients.push_back(clients[i]);
    const uint8_t *b = reinterpret_cast<const uint8_t *>(progs[i]);
    p->code.emplace_back(b, b + lens[i] * sizeof(ce_insn));
    if (std::find(p->regfiles.begin(), p->regfiles.end(), clients[i]) == p->regfiles.end())
      p->regfiles.push_back(clients[i]);
  }
  const size_t nrf = p->regfiles.size();
  ce_status s = E.reserve(E.next_slot + nrf * kRegBits + 1);
  if (s != CE_OK) return s;
  p->in_base = uint32_t(E.next_slot);
  for (size_t k = 0; k < nrf * kRegBits; ++k) {
    const uint32_t sl = uint32_t(E.next_slot++);
    if (E.rc.size() <= sl) E.rc.resize(sl + 1, 0);
    E.rc[sl] = 1;  // owned by the plan
    p->slots.push_back(sl);
  }
  // simulated register files over the input slots (one reference each)
  std::vector<RegFile> rf(nrf);
  for (size_t u = 0; u < nrf; ++u) {
    const uint32_t base = p->in_base + uint32_t(u * kRegBits);
    for (int j = 0; j < kRegs; ++j)
      for (int b = 0; b < kWidth; ++b) {
        rf[u].r[j][b] = SRef{base + uint32_t(j * kWidth + b), false};
        E.ref(rf[u].r[j][b]);
      }
    for (int k = 0; k < 4; ++k) {
      rf[u].nzcv[k] = SRef{base + uint32_t(kRegs * kWidth + k), false};
      E.ref(rf[u].nzcv[k]);
    }
  }
  auto release_rf = [&] {
    for (RegFile &R : rf) {
      for (auto &reg : R.r)
        for (auto &b : reg) E.unref(b);
      for (auto &b : R.nzcv) E.unref(b);
    }
  };
  std::vector<Run> runs(n_prog);
  for (size_t i = 0; i < n_prog; ++i) {
    runs[i].client = clients[i];
    runs[i].code = progs[i];
    runs[i].n = lens[i];
    runs[i].rf = &rf[std::find(p->regfiles.begin(), p->regfiles.end(), clients[i]) -
                     p->regfiles.begin()];
  }
  std::vector<uint8_t> blob;
  auto fail = [&](ce_status st) {
    for (Run &r : runs)
      if (r.cur) {
        if (!r.cur->wire.empty()) E.complete(*r.cur);
        for (const SRef &x : r.cur->result) E.unref(x);
      }
    release_rf();
    E.drop_prog_plan(*p);
    return st;
  };
  for (;;) {
    std::vector<Instance *> act;
    for (Run &r : runs) {
      s = advance(E, r);
      if (s != CE_OK) return fail(s);
      if (r.cur) act.push_back(r.cur.get());
    }
    if (act.empty()) break;
    TickDesc t;
    s = E.build_tick(act, t);
    if (s != CE_OK) return fail(s);
    p->max_jobs = std::max(p->max_jobs, t.jobs.size());
    p->levels.push_back(E.record_level(t, blob, p->slots));
    ++p->ticks;
    for (Instance *in : act) ++in->level;
    for (Run &r : runs)
      if (r.cur && r.cur->level == r.cur->net->depth) retire(E, r);
  }
  // the plan keeps the final register references, the simulation lets go
  for (size_t u = 0; u < nrf; ++u) {
    std::vector<SRef> refs;
    for (int j = 0; j < kRegs; ++j)
      for (int b = 0; b < kWidth; ++b) refs.push_back(rf[u].r[j][b]);
    for (int k = 0; k < 4; ++k) refs.push_back(rf[u].nzcv[k]);
    for (const SRef &r : refs) {
      E.ref(r);
      if (r.slot > kSlotSink) ++p->n_out_copies;
    }
    p->final_refs.push_back(refs);
  }
  release_rf();
  cudaError_t e = cudaSuccess;
  if (!blob.empty()) {
    e = dev_malloc(&p->d_desc, blob.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(p->d_desc, blob.data(), blob.size(), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = dev_malloc(&p->d_map, (nrf * kRegBits + p->n_out_copies) * 3 * sizeof(uint32_t));
  if (e != cudaSuccess) return fail(cuda_error(e, "program plan upload"));
  if (E.pplans.size() >= 8) {  // evict the least recently used program plan
    auto lru = std::min_element(E.pplans.begin(), E.pplans.end(), [](const auto &a, const auto &b) {
      return a->last_use < b->last_use;
    });
    E.drop_prog_plan(**lru);
    E.pplans.erase(lru);
  }
  *out = p.get();
  E.pplans.push_back(std::move(p));
  return CE_OK;
}

// Enqueues the copy-in, the recorded ticks and the copy-out of a plan.
ce_status launch_prog_plan(Engine &E, ProgPlan &p, cudaStream_t st, int *launches) {
  const size_t n_in = p.regfiles.size() * kRegBits;
  copy_slots_kernel<<<unsigned(n_in), 128, 0, st>>>(p.d_map, E.arena);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "program copy-in");
  ++*launches;
  ce_status s = E.launch_levels(p.levels, p.d_desc, st, launches);
  if (s != CE_OK) return s;
  if (p.n_out_copies) {
    copy_slots_kernel<<<unsigned(p.n_out_copies), 128, 0, st>>>(p.d_map + 3 * n_in, E.arena);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "program copy-out");
    ++*launches;
  }
  return CE_OK;
}

// One run of a planned program set on the clients' current registers:
// fresh slots receive the final register bits; the register files then
// point at them.  The ticks replay as the plan's captured graph.
ce_status run_prog_plan(Engine &E, ProgPlan &p, cudaStream_t st, int *launches) {
  ce_ctx *ctx = E.ctx;
  ce_status s = ensure_job_scratch(ctx, p.max_jobs);
  if (s != CE_OK) return s;
  const size_t nrf = p.regfiles.size();
  std::vector<uint32_t> map;
  map.reserve((nrf * kRegBits + p.n_out_copies) * 3);
  for (size_t u = 0; u < nrf; ++u) {
    const RegFile &R = E.regs(p.regfiles[u]);
    const uint32_t base = p.in_base + uint32_t(u * kRegBits);
    for (int k = 0; k < kRegBits; ++k) {
      const SRef &x = k < kRegs * kWidth ? R.r[k / kWidth][k % kWidth] : R.nzcv[k - kRegs * kWidth];
      map.insert(map.end(), {x.slot, x.neg ? 1u : 0u, base + uint32_t(k)});
    }
  }
  std::vector<std::vector<SRef>> fresh(nrf);  // the registers' new references
  for (size_t u = 0; u < nrf; ++u)
    for (const SRef &r : p.final_refs[u]) {
      if (r.slot <= kSlotSink) {  // constants stay constants
        fresh[u].push_back(r);
        continue;
      }
      uint32_t sl;
      s = E.alloc(&sl);
      if (s != CE_OK) {
        for (auto &f : fresh)
          for (const SRef &x : f) E.unref(x);
        return s;
      }
      fresh[u].push_back(SRef{sl, false});
      map.insert(map.end(), {r.slot, r.neg ? 1u : 0u, sl});
    }
  // pageable source: the copy is complete for the host when the call returns
  cudaError_t e = cudaMemcpyAsync(p.d_map, map.data(), map.size() * sizeof(uint32_t),
                                  cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "program map upload");
  if (p.exec && p.exec_gen != ctx->scratch_gen) E.drop_prog_graph(p);  // scratch replaced
  if (!p.exec) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(E.cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_error(e, "begin capture");
    int cnt = 0;
    s = launch_prog_plan(E, p, E.cap_stream, &cnt);
    e = cudaStreamEndCapture(E.cap_stream, &g);
    if (s != CE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "program graph instantiate");
    p.graph_launches = cnt;
    p.exec_gen = ctx->scratch_gen;
  }
  e = cudaGraphLaunch(p.exec, st);
  if (e != cudaSuccess) return cuda_error(e, "program graph launch");
  *launches += p.graph_launches;
  for (size_t u = 0; u < nrf; ++u) {
    RegFile &R = E.regs(p.regfiles[u]);
    for (int k = 0; k < kRegBits; ++k) {
      SRef &x = k < kRegs * kWidth ? R.r[k / kWidth][k % kWidth] : R.nzcv[k - kRegs * kWidth];
      E.unref(x);
      x = fresh[u][k];
      if (x.slot <= kSlotSink) E.ref(x);
    }
  }
  p.last_use = ++E.use_clock;
  return CE_OK;
}

}  // namespace

void serve_runs_forget(Engine *e) {
  auto it = g_serve_runs.find(e);
  if (it == g_serve_runs.end()) return;
  for (auto &kv : it->second)
    if (kv.second.cur) {
      e->complete(*kv.second.cur);
      for (const SRef &x : kv.second.cur->result) e->unref(x);
    }
  g_serve_runs.erase(it);
}

int gates_at_level(const Instance &in) {
  const Netlist &n = *in.net;
  int k = 0;
  for (int g = n.level_begin[in.level]; g < n.level_begin[in.level + 1]; ++g)
    k += n.gates[g].op == kOpMux ? 2 : 1;
  return k;
}

ce_status engine_serve_tick(ce_ctx *ctx, cudaStream_t st, const std::vector<int> &start_clients,
                            const std::vector<ce_insn> &start_insns, std::vector<int> &retired,
                            int *active_after, int *bootstraps) {
  CtxWork work(ctx, st);
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  auto &runs = g_serve_runs[E];
  for (size_t i = 0; i < start_clients.size(); ++i) {
    Run &r = runs[start_clients[i]];
    r = Run();
    r.client = start_clients[i];
    r.one = start_insns[i];
    r.code = &r.one;
    r.n = 1;
    s = advance(*E, r);
    if (s != CE_OK) {
      runs.erase(start_clients[i]);
      return s;
    }
    if (!r.cur) {  // no bootstrap needed: done now
      retired.push_back(r.client);
      runs.erase(start_clients[i]);
    }
  }
  std::vector<Instance *> act;
  int boots = 0;
  for (auto &kv : runs) {
    act.push_back(kv.second.cur.get());
    boots += gates_at_level(*kv.second.cur);
  }
  if (!act.empty()) {
    int launches = 0;
    s = E->tick(act, st, &launches);
    if (s != CE_OK) return s;
  }
  for (auto it = runs.begin(); it != runs.end();) {
    if (it->second.cur->level == it->second.cur->net->depth) {
      retire(*E, it->second);
      retired.push_back(it->first);
      it = runs.erase(it);
    } else {
      ++it;
    }
  }
  *active_after = int(runs.size());
  *bootstraps = boots;
  return CE_OK;
}

ce_status exec_programs(ce_ctx *ctx, size_t n_prog, const int *clients, const ce_insn *const *progs,
                        const size_t *lens, uint64_t timeout_ns, cudaStream_t st, int *ticks) {
  CtxWork work(ctx, st);
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  std::vector<Run> runs(n_prog);
  for (size_t i = 0; i < n_prog; ++i) {
    if (!live_client(ctx, clients[i])) return set_error(CE_ENOTFOUND, "ce_exec: unknown client");
    if (lens[i] && !progs[i]) return set_error(CE_EINVAL, "ce_exec: null program");
    runs[i].client = clients[i];
    runs[i].code = progs[i];
    runs[i].n = lens[i];
  }
  *ticks = 0;
  if (E->use_graphs && !ctx->profile && E->trace_per_tick == 0 && timeout_ns == 0) {
    // planned once per program set, replayed as a captured graph (a host
    // time limit needs the eager tick loop, which checks it between ticks)
    ProgPlan *p = nullptr;
    for (auto &pp : E->pplans)
      if (plan_matches(ctx, *pp, n_prog, clients, progs, lens)) p = pp.get();
    if (!p) {
      s = make_prog_plan(*E, n_prog, clients, progs, lens, &p);
      if (s != CE_OK) return s;
    }
    int launches = 0;
    s = run_prog_plan(*E, *p, st, &launches);
    if (s != CE_OK) return s;
    *ticks = p->ticks;
    ctx->last_launches = launches;
    return CE_OK;
  }
  const auto t0 = std::chrono::steady_clock::now();
  int launches = 0;
  // On an error return, release what unfinished instructions hold.
  struct Cleanup {
    Engine *E;
    std::vector<Run> *runs;
    ~Cleanup() {
      for (Run &r : *runs)
        if (r.cur) {
          if (!r.cur->wire.empty()) E->complete(*r.cur);
          for (const SRef &x : r.cur->result) E->unref(x);
          r.cur.reset();
        }
    }
  } cleanup{E, &runs};
  for (;;) {
    std::vector<Instance *> act;
    for (Run &r : runs) {
      s = advance(*E, r);
      if (s != CE_OK) return s;
      if (r.cur) act.push_back(r.cur.get());
    }
    if (act.empty()) break;
    s = E->tick(act, st, &launches);
    if (s != CE_OK) return s;
    ++*ticks;
    for (Run &r : runs)
      if (r.cur && r.cur->level == r.cur->net->depth) retire(*E, r);
    if (timeout_ns) {
      const auto dt = std::chrono::steady_clock::now() - t0;
      if (uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(dt).count()) > timeout_ns)
        return set_error(CE_ETIMEOUT, "ce_exec: timeout");
    }
  }
  ctx->last_launches = launches;
  return CE_OK;
}

}  // namespace ce

using namespace ce;

extern "C" ce_status ce_unit_eval_device_width(ce_ctx *ctx, int client, int unit, int cond,
                                               int width, const uint32_t *d_in, uint32_t *d_out,
                                               size_t n, void *cuda_stream) {
  if (!ctx) return set_error(CE_EINVAL, "ce_unit_eval_device: null context");
  if (unit < 0 || unit >= kUnitCount || cond < 0 || cond > 13)
    return set_error(CE_EINVAL, "ce_unit_eval_device: bad unit or condition");
  if (width < 2 || width > 32 || (width & (width - 1)))
    return set_error(CE_EINVAL, "ce_unit_eval_device: width must be a power of two in 2..32");
  cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->stream;
  CtxWork work(ctx, st);
  if (!live_client(ctx, client)) return set_error(CE_ENOTFOUND, "ce_unit_eval_device: unknown client");
  if (n == 0) {
    ctx->last_launches = 0;
    return CE_OK;
  }
  if (!d_in || !d_out) return set_error(CE_EINVAL, "ce_unit_eval_device: null buffer");
  if (n > (size_t(1) << 20)) return set_error(CE_EINVAL, "ce_unit_eval_device: n too large");
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  int launches = 0;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  s = E->eval_unit(unit, cond, width, client, d_in, d_out, n, st, &launches);
  ctx->last_launches = launches;
  return s;
}

extern "C" ce_status ce_unit_eval(ce_ctx *ctx, int client, int unit, int cond, int width,
                                  const ce_lwe *in, ce_lwe *out, size_t n) {
  if (!ctx) return set_error(CE_EINVAL, "ce_unit_eval: null context");
  if (unit < 0 || unit >= kUnitCount || cond < 0 || cond > 13)
    return set_error(CE_EINVAL, "ce_unit_eval: bad unit or condition");
  if (width < 2 || width > 32 || (width & (width - 1)))
    return set_error(CE_EINVAL, "ce_unit_eval: width must be a power of two in 2..32");
  if (n && (!in || !out)) return set_error(CE_EINVAL, "ce_unit_eval: null buffer");
  if (n > (size_t(1) << 20)) return set_error(CE_EINVAL, "ce_unit_eval: n too large");
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  CtxWork work(ctx, st);
  if (!live_client(ctx, client)) return set_error(CE_ENOTFOUND, "ce_unit_eval: unknown client");
  if (n == 0) {
    ctx->last_launches = 0;
    return CE_OK;
  }
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  const Netlist *net = E->netlist(unit, cond, width);
  if (!net) return set_error(CE_EINVAL, "ce_unit_eval: bad unit or width");
  const size_t in_bytes = n * net->n_inputs * sizeof(ce_lwe);
  const size_t out_bytes = n * net->outputs.size() * sizeof(ce_lwe);
  s = E->ensure_unit_io(in_bytes, out_bytes);
  if (s != CE_OK) return s;
  cudaError_t e = cudaMemcpyAsync(E->io_in, in, in_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_error(e, "ce_unit_eval upload");
  int launches = 0;
  s = E->eval_unit(unit, cond, width, client, E->io_in, E->io_out, n, st, &launches);
  if (s != CE_OK) return s;
  ctx->last_launches = launches;
  e = cudaMemcpyAsync(out, E->io_out, out_bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_error(e, "ce_unit_eval");
  return check_device_error(ctx);
}

extern "C" ce_status ce_unit_eval_device(ce_ctx *ctx, int client, int unit, int cond,
                                         const uint32_t *d_in, uint32_t *d_out, size_t n,
                                         void *cuda_stream) {
  return ce_unit_eval_device_width(ctx, client, unit, cond, 16, d_in, d_out, n, cuda_stream);
}

extern "C" ce_status ce_set_instruction_circuits(ce_ctx *ctx, int low_latency) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_instruction_circuits: null context");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  ctx->fast_circuits = low_latency != 0;
  return CE_OK;
}

extern "C" ce_status ce_set_level_batching(ce_ctx *ctx, int on) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_level_batching: null context");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  ctx->per_gate = on == 0;
  return CE_OK;
}

extern "C" ce_status ce_set_unit_graphs(ce_ctx *ctx, int on) {
  if (!ctx) return set_error(CE_EINVAL, "ce_set_unit_graphs: null context");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  E->use_graphs = on != 0;
  return CE_OK;
}

extern "C" ce_status ce_reg_write(ce_ctx *ctx, int client, int reg, const ce_lwe *bits) {
  if (!ctx || !bits || reg < 0 || reg >= kRegs) return set_error(CE_EINVAL, "ce_reg_write: bad argument");
  CtxWork work(ctx, ctx->stream);
  if (!live_client(ctx, client)) return set_error(CE_ENOTFOUND, "ce_reg_write: unknown client");
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  RegFile &R = E->regs(client);
  uint32_t sl[kWidth];
  for (int j = 0; j < kWidth; ++j) {
    s = E->alloc(&sl[j]);
    if (s != CE_OK) return s;
  }
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < kWidth && e == cudaSuccess; ++j)
    e = cudaMemcpyAsync(E->arena + size_t(sl[j]) * kSlotWords, &bits[j], sizeof(ce_lwe),
                        cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  for (int j = 0; j < kWidth; ++j) {
    E->unref(R.r[reg][j]);
    R.r[reg][j] = SRef{sl[j], false};
  }
  return e == cudaSuccess ? CE_OK : cuda_error(e, "ce_reg_write");
}

static ce_status read_refs(ce_ctx *ctx, Engine *E, const SRef *refs_in, int count, ce_lwe *out) {
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  SRef refs[kWidth];
  for (int j = 0; j < count; ++j) refs[j] = refs_in[j];
  // Device-wide: the slots may have been written on a serving loop's stream.
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  for (int j = 0; j < count && e == cudaSuccess; ++j)
    e = cudaMemcpy(&out[j], E->arena + size_t(refs[j].slot) * kSlotWords, sizeof(ce_lwe),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "register read");
  for (int j = 0; j < count; ++j)
    if (refs[j].neg) {
      for (int m = 0; m < kLweN; ++m) out[j].a[m] = 0u - out[j].a[m];
      out[j].b = 0u - out[j].b;
    }
  return CE_OK;
}

extern "C" ce_status ce_reg_read(ce_ctx *ctx, int client, int reg, ce_lwe *bits) {
  if (!ctx || !bits || reg < 0 || reg >= kRegs) return set_error(CE_EINVAL, "ce_reg_read: bad argument");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  if (!live_client(ctx, client)) return set_error(CE_ENOTFOUND, "ce_reg_read: unknown client");
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  return read_refs(ctx, E, E->regs(client).r[reg], kWidth, bits);
}

extern "C" ce_status ce_flags_read(ce_ctx *ctx, int client, ce_lwe *nzcv) {
  if (!ctx || !nzcv) return set_error(CE_EINVAL, "ce_flags_read: bad argument");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  if (!live_client(ctx, client)) return set_error(CE_ENOTFOUND, "ce_flags_read: unknown client");
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  return read_refs(ctx, E, E->regs(client).nzcv, 4, nzcv);
}

extern "C" ce_status ce_exec(ce_ctx *ctx, int client, const ce_insn *prog, size_t n,
                             uint64_t timeout_ns) {
  if (!ctx) return set_error(CE_EINVAL, "ce_exec: null context");
  int ticks = 0;
  return exec_programs(ctx, 1, &client, &prog, &n, timeout_ns, ctx->stream, &ticks);
}

extern "C" ce_status ce_exec_multi(ce_ctx *ctx, size_t n_programs, const int *clients,
                                   const ce_insn *const *progs, const size_t *lens,
                                   uint64_t timeout_ns) {
  if (!ctx || (n_programs && (!clients || !progs || !lens)))
    return set_error(CE_EINVAL, "ce_exec_multi: bad argument");
  int ticks = 0;
  return exec_programs(ctx, n_programs, clients, progs, lens, timeout_ns, ctx->stream, &ticks);
}

extern "C" ce_status ce_trace_enable(ce_ctx *ctx, int per_tick, size_t cap) {
  if (!ctx) return set_error(CE_EINVAL, "ce_trace_enable: null context");
  if (per_tick < 0 || per_tick > 4096 || (per_tick > 0 && (cap == 0 || cap > (size_t(1) << 20))))
    return set_error(CE_EINVAL, "ce_trace_enable: per_tick must lie in 0..4096 and cap in "
                                "1..2^20");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();  // records of earlier ticks may still be in flight
  dev_free(E->trace_rec);
  dev_free(E->trace_count);
  E->trace_rec = nullptr;
  E->trace_count = nullptr;
  E->trace_cap = 0;
  E->trace_per_tick = 0;
  E->trace_tick = 0;
  if (per_tick == 0) return CE_OK;
  cudaError_t e = dev_malloc(&E->trace_rec, cap * sizeof(ce_trace_rec));
  if (e == cudaSuccess) e = dev_malloc(&E->trace_count, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(E->trace_count, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    dev_free(E->trace_rec);
    dev_free(E->trace_count);
    E->trace_rec = nullptr;
    E->trace_count = nullptr;
    return set_error(CE_ENOMEM, "ce_trace_enable: record buffer allocation failed");
  }
  E->trace_cap = cap;
  E->trace_per_tick = per_tick;
  return CE_OK;
}

extern "C" ce_status ce_trace_read(ce_ctx *ctx, ce_trace_rec *out, size_t cap, size_t *count,
                                   uint64_t *seen) {
  if (!ctx || !count || (cap && !out)) return set_error(CE_EINVAL, "ce_trace_read: bad argument");
  std::lock_guard<std::recursive_mutex> ctx_lock(ctx->mu);
  Engine *E;
  ce_status s = get_engine(ctx, &E);
  if (s != CE_OK) return s;
  std::lock_guard<std::recursive_mutex> lock(E->mu);
  *count = 0;
  if (seen) *seen = 0;
  if (!E->trace_count) return CE_OK;
  cudaSetDevice(ctx->device);
  unsigned long long total = 0;
  cudaError_t e = cudaDeviceSynchronize();  // ticks may have run on any stream
  if (e == cudaSuccess)
    e = cudaMemcpy(&total, E->trace_count, sizeof(total), cudaMemcpyDeviceToHost);
  const size_t stored = size_t(std::min<unsigned long long>(total, E->trace_cap));
  const size_t n = std::min(stored, cap);
  if (e == cudaSuccess && n)
    e = cudaMemcpy(out, E->trace_rec, n * sizeof(ce_trace_rec), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(E->trace_count, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_error(e, "ce_trace_read");
  *count = n;
  if (seen) *seen = total;
  return CE_OK;
}

extern "C" ce_status ce_exec_branching(ce_ctx *ctx, int client, const ce_insn *prog, size_t n,
                                       ce_branch_fn decide, void *user, uint64_t max_steps,
                                       uint64_t timeout_ns, uint64_t *steps_out) {
  if (steps_out) *steps_out = 0;
  if (!ctx || (n && !prog) || !decide)
    return set_error(CE_EINVAL, "ce_exec_branching: bad argument");
  if (n > 256) return set_error(CE_EINVAL, "ce_exec_branching: at most 256 instructions");
  for (size_t i = 0; i < n; ++i)
    if ((prog[i].op == kB || prog[i].op == kBcond) && prog[i].imm > n)
      return set_error(CE_EINVAL, "ce_exec_branching: branch target beyond the program end");
  const auto t0 = std::chrono::steady_clock::now();
  auto left_ns = [&]() -> uint64_t {
    if (!timeout_ns) return 0;
    const uint64_t dt = uint64_t(std::chrono::duration_cast<std::chrono::nanoseconds>(
                                     std::chrono::steady_clock::now() - t0)
                                     .count());
    return dt >= timeout_ns ? 1 : timeout_ns - dt;
  };
  uint64_t steps = 0;
  size_t pc = 0;
  while (pc < n) {
    // straight-line run up to the next branch: one program of the engine
    size_t end = pc;
    while (end < n && prog[end].op != kB && prog[end].op != kBcond) ++end;
    if (max_steps && steps + (end - pc) > max_steps)
      return set_error(CE_ETIMEOUT, "ce_exec_branching: step limit reached");
    if (end > pc) {
      const ce_insn *seg = prog + pc;
      const size_t len = end - pc;
      int ticks = 0;
      ce_status s = exec_programs(ctx, 1, &client, &seg, &len, left_ns(), ctx->stream, &ticks);
      if (s != CE_OK) return s;
      steps += len;
      pc = end;
      if (steps_out) *steps_out = steps;
    }
    if (pc == n) break;
    if (max_steps && steps + 1 > max_steps)
      return set_error(CE_ETIMEOUT, "ce_exec_branching: step limit reached");
    const ce_insn &I = prog[pc];
    bool taken = true;
    if (I.op == kBcond) {
      if (I.cond > 13) return set_error(CE_EINVAL, "ce_exec_branching: bad condition");
      // the cloud hands the encrypted flags and the condition to the key
      // owner, who returns the decision; no context lock is held meanwhile
      ce_lwe nzcv[4];
      ce_status s = ce_flags_read(ctx, client, nzcv);
      if (s != CE_OK) return s;
      const int d = decide(user, client, I.cond, nzcv);
      if (d < 0) return set_error(CE_EINVAL, "ce_exec_branching: the branch decision failed");
      taken = d != 0;
    }
    pc = taken ? size_t(I.imm) : pc + 1;
    ++steps;
    if (steps_out) *steps_out = steps;
    if (timeout_ns && left_ns() == 1) return set_error(CE_ETIMEOUT, "ce_exec_branching: timeout");
  }
  return CE_OK;
}
