/*
 * cryptoemu.h — C ABI of the GB300 TFHE gate-bootstrapping library.
 *
 * The library evaluates the bootstrapped binary gates on which the paper's
 * homomorphic functional units are built (§3 "TFHE Library", Table "TFHE API
 * Benchmark": NAND, OR, AND, XOR, XNOR, NOR, ANDNY, ANDYN, ORNY, ORYN and
 * MUX; one bootstrap per binary gate, two for MUX).  A gate is four steps:
 * the linear LWE combination, the modulus switch to 2N, blind rotation
 * (n = 500 CMux external products over Z_{2^32}[X]/(X^1024 + 1)) and sample
 * extraction followed by LWE key switching.  The client side (keygen, encrypt,
 * decrypt) follows the paper's cloud service model (§4, "Cloud service
 * model"): the secret key stays in memory the client owns; the cloud key
 * (bootstrapping + key-switching key) is handed to a context that keeps it
 * resident on the GPU.
 *
 * Parameters (fixed): LWE n = 500, sigma = 2^-15; TRLWE N = 1024, k = 1;
 * gadget l = 3, Bg = 2^10, sigma_bk = 9e-9; key switch t = 8, base 2^2.
 * Torus values are uint32 (x <-> x / 2^32); a bit is encoded as +1/8 (true)
 * or -1/8 (false).  All GPU arithmetic is exact integer arithmetic, so every
 * result is bit-identical to the plain CPU definition of the same step.
 *
 * Conventions for every call:
 *  - Returns a ce_status (0 = success); nothing aborts the process.  On error
 *    ce_last_error() returns a message for the calling thread.
 *  - Host buffers are owned by the caller and only read/written during the
 *    call.  Device buffers ("_device" calls) are owned by the caller, must
 *    live on the context's device and stay valid until the work enqueued on
 *    the given stream has finished; those calls are asynchronous.
 *  - Everything the context allocates on the device (keys, scratch) is owned
 *    by the context and released by ce_destroy / ce_client_evict.
 *  - Calls on one context may come from several host threads (a serving
 *    loop's worker is one): the calls that enqueue GPU work take the
 *    context's lock, and each one's GPU work is ordered after the previous
 *    one's, whichever stream either used.  ce_destroy must not race with any
 *    other call on the context, and needs every serving loop destroyed first.
 */
#ifndef CRYPTOEMU_H
#define CRYPTOEMU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CE_LWE_N 500          /* LWE dimension n */
#define CE_LWE_WORDS 501      /* words of one LWE ciphertext: a[500], b */
#define CE_RING_N 1024        /* TRLWE ring degree N */
#define CE_BSK_WORDS (500u * 6u * 2u * 1024u)        /* 3,072,000 uint32 */
#define CE_KSK_WORDS (1024u * 8u * 4u * 501u)        /* 16,416,768 uint32 */

/* Status of every call (the paper's emulator has no error model; these are
 * this library's). */
typedef enum {
    CE_OK = 0,
    CE_EINVAL = -1,     /* bad argument (null pointer, size, opcode, id) */
    CE_ENOMEM = -2,     /* host or device allocation failed */
    CE_EADMIT = -3,     /* client refused: over the context's HBM budget */
    CE_ETIMEOUT = -4,   /* a bounded device-side wait or a timeout expired */
    CE_ECUDA = -5,      /* CUDA runtime error (no device, launch failure, ...) */
    CE_ENOTFOUND = -6   /* unknown client id */
} ce_status;

/* Bootstrapped binary gates (truth tables: §3, Table "TFHE API Benchmark").
 * ANDNY(a,b) = (NOT a) AND b, ANDYN(a,b) = a AND (NOT b), ORNY, ORYN alike. */
typedef enum {
    CE_NAND = 0, CE_AND = 1, CE_OR = 2, CE_XOR = 3, CE_NOR = 4, CE_XNOR = 5,
    CE_ANDNY = 6, CE_ANDYN = 7, CE_ORNY = 8, CE_ORYN = 9
} ce_gate_op;

/* One LWE ciphertext (§3 "TFHE Library": the encrypted bit every gate takes
 * and returns): 2004 bytes, a[0..499] then b. */
typedef struct { uint32_t a[CE_LWE_N]; uint32_t b; } ce_lwe;

/* The cloud side of §4 "Cloud service model": holds the admitted clients'
 * cloud keys on the GPU, their encrypted register files and scratch. */
typedef struct ce_ctx ce_ctx;

/* ------------------------------------------------------------- client --- */

/* Secret key bytes: "CESK" magic (4 B), version (uint32 = 1), then the LWE key
 * s[500] and the TRLWE key K[1024] as uint32 values in {0,1}.  Each bit is the
 * top bit of one uniform draw of the counter-based SplitMix64 stream
 * described in ce_cloud_keygen.  The buffer is allocated by the library and
 * freed with ce_free.  (§4 "Cloud service model": the user owns the secret
 * key; §3: the TFHE library's key generation.) */
#define CE_SECRET_BYTES (8u + 4u * (500u + 1024u))
ce_status ce_secret_keygen(uint64_t seed, void **secret_out, size_t *bytes_out);

/* Cloud key bytes: "CECK" magic, version (uint32 = 1), then the bootstrapping
 * key BSK[i][r][comp][j] (i < 500 key bits, r = c*3 + (p-1) TRGSW rows with
 * c = 0 a-part / 1 b-part and p = 1..3 gadget levels, comp 0 = a / 1 = b,
 * j < 1024 coefficients; each row a TRLWE encryption of zero under K with
 * s_i * 2^(32 - 10 p) added to the constant coefficient of component c), then
 * the key-switching key KSK[j][q][v][m] (j < 1024, q < 8, v < 4, m <= 500; an
 * LWE encryption under s of v * K_j * 2^(32 - 2 (q+1)); v = 0 rows stored).
 * Randomness: uniform draw i of domain d is the high half of SplitMix64
 * output d * 2^40 + i for the given seed; Gaussian noise i uses draws 2i and
 * 2i+1 through Box-Muller (domains: 3 BSK a, 4 BSK noise, 5 KSK a, 6 KSK
 * noise).  Allocated by the library (about 78 MB), freed with ce_free.
 * The TRGSW construction is the one of the TFHE papers cited in §2/§3. */
#define CE_CLOUD_BYTES (8ull + 4ull * ((unsigned long long)CE_BSK_WORDS + CE_KSK_WORDS))
ce_status ce_cloud_keygen(const void *secret, uint64_t seed, void **cloud_out,
                          size_t *bytes_out);
void ce_free(void *p);

/* Encrypt one bit: a[m] = uniform draw ctr*500 + m of domain 7, b = <a,s> +
 * e + (bit ? +1/8 : -1/8), e = Gaussian draw ctr of domain 8 (sigma 2^-15).
 * (§3, Table "TFHE API Benchmark": Encrypt.) */
ce_status ce_encrypt_bit(const void *secret, int bit, uint64_t seed,
                         uint64_t ctr, ce_lwe *out);
/* Decrypt: returns 1 if b - <a,s> read as a signed 32-bit value is > 0, 0
 * otherwise, or a negative ce_status on a bad argument.  (§3: Decrypt.) */
int ce_decrypt_bit(const void *secret, const ce_lwe *c);

/* ------------------------------------------------------------- context --- */

/* Create a context on CUDA device `device` (§4 "Cloud service model": the
 * cloud that evaluates instructions over its users' encrypted data).
 * `hbm_budget_bytes` caps the device memory the context's clients may hold
 * (0 = 90% of the free memory at creation).  `cuda_stream` (a cudaStream_t,
 * may be NULL for the legacy default stream) is the stream all synchronous
 * calls enqueue on.  CE_ECUDA without a device, CE_EINVAL for a bad index. */
ce_status ce_create(ce_ctx **out, int device, uint64_t hbm_budget_bytes,
                    void *cuda_stream);
/* Waits for all work on the device, then frees everything the context owns
 * (keys, registers, scratch).  NULL is ignored. */
void ce_destroy(ce_ctx *ctx);
/* Message of the calling thread's last failed call (this library's error
 * model; the paper has none).  Valid until that thread's next failing call. */
const char *ce_last_error(void);
/* Device allocations (cudaMalloc) and frees the library has made in this
 * process, for callers that budget device memory and for tests (the paper
 * has no counterpart).  Either pointer may be NULL. */
void ce_device_alloc_count(uint64_t *allocations, uint64_t *frees);

/* Admit a client (§4 "Cloud service model": a user hands the cloud the
 * public material its homomorphic evaluation needs): copies its cloud key
 * (CE_CLOUD_BYTES host bytes, caller-owned, read during the call) to the
 * device and converts the bootstrapping key to the negacyclic-transform
 * domain used by the blind-rotation kernel (98,304 B per key bit); the
 * coefficient key stays resident too (for the tensor-core external product).
 * Returns CE_EADMIT when the client's device footprint would exceed the
 * budget, CE_EINVAL for bytes that are not a cloud key. */
ce_status ce_client_admit(ce_ctx *ctx, const void *cloud_key, size_t bytes,
                          int *client_id);
/* Evict a client (§4: the user leaves the cloud): waits for all work on the
 * device, then frees its keys, registers and cached unit plans.
 * CE_ENOTFOUND for an unknown id; CE_EINVAL while a serving loop has one of
 * its requests queued or running (wait for them first). */
ce_status ce_client_evict(ce_ctx *ctx, int client_id);
/* Device bytes a client holds at admission (keys + register file; the
 * tensor-core external product adds its key form on first use). */
uint64_t ce_client_footprint_bytes(void);

/* ---------------------------------------------------------------- gates --- */

/* One bootstrapped gate out = op(a, b) with host ciphertexts (blocking):
 * one of the bootstrapped gates of §3, Table "TFHE API Benchmark".
 * CE_EINVAL for a bad opcode or NULL buffer, CE_ENOTFOUND for an unknown
 * client. */
ce_status ce_gate(ce_ctx *ctx, int client, ce_gate_op op, const ce_lwe *a,
                  const ce_lwe *b, ce_lwe *out);
/* n independent gates out[i] = ops[i](a[i], b[i]) with host buffers (§3,
 * Table "TFHE API Benchmark", batched as the independent gates of §5's
 * OpenMP sections): copies the inputs to the device, runs the batched path
 * and copies the results back (blocking).  ops: n bytes (ce_gate_op
 * values). */
ce_status ce_gates_batch(ce_ctx *ctx, int client, const uint8_t *ops,
                         const ce_lwe *a, const ce_lwe *b, ce_lwe *out, size_t n);
/* Same on device buffers (d_ops: n bytes; d_a, d_b, d_out: n x 501 uint32,
 * packed), enqueued on `cuda_stream` (NULL = the context's stream) without
 * host synchronisation.  Steps: linear combination + modulus switch, blind
 * rotation (one persistent launch for all n gates, bootstrapping key staged
 * through shared memory and shared by the gates of a block), fused sample
 * extraction + key switching.  Scratch (10 KB per gate) is owned by the
 * context and grows on demand. */
ce_status ce_gates_batch_device(ce_ctx *ctx, int client, const uint8_t *d_ops,
                                const uint32_t *d_a, const uint32_t *d_b,
                                uint32_t *d_out, size_t n, void *cuda_stream);

/* n MUX gates out[i] = a[i] ? b[i] : c[i] on device buffers (two bootstraps
 * without key switching and one key switch per MUX; §3: MUX is bootstrapped
 * twice). */
ce_status ce_mux_batch_device(ce_ctx *ctx, int client, const uint32_t *d_a,
                              const uint32_t *d_b, const uint32_t *d_c,
                              uint32_t *d_out, size_t n, void *cuda_stream);

/* Building block of the blind rotation, exposed for verification: n exact
 * negacyclic products out[i] = d[i] * k[i] in Z_{2^32}[X]/(X^1024 + 1), d a
 * polynomial of signed 16-bit coefficients in [-8192, 8192] (the blind
 * rotation's digits lie in [-512, 511]), k of uint32 coefficients (taken as
 * signed), through the same two-prime 1024-point transform the blind
 * rotation uses (primes 2^28 - 2^16 + 1 and 2^28 - 2^16 - 2^11 + 1; exact
 * because |sum| <= 1024 * 2^13 * 2^31 = 2^54 < p0 p1 / 2; coefficients of d
 * outside that range give unspecified results).  Device buffers
 * d_d (n x 1024 int16), d_k, d_out (n x 1024 uint32); asynchronous. */
ce_status ce_negacyclic_mul_device(ce_ctx *ctx, const int16_t *d_d,
                                   const uint32_t *d_k, uint32_t *d_out,
                                   size_t n, void *cuda_stream);

/* Tuning of the blind-rotation launch: gates per block (1, 2 or 4, or 3 for
 * the latency shape: one gate per block whose three thread groups transform
 * the three gadget levels concurrently) and resident blocks per SM; 0 =
 * autotuned choice.  Applies to later calls. */
ce_status ce_set_blind_rotate_config(ce_ctx *ctx, int gates_per_block,
                                     int blocks_per_sm);
/* The launches a blind rotation of n_jobs gates makes in shape
 * gates_per_block (1-4 as above) over `blocks` blocks (no paper passage:
 * launch planning, callable without a GPU).  When the gate groups leave the
 * last round over the blocks part filled (shapes 2 and 4), the whole rounds
 * run as one launch and the remaining gates as a second one with fewer gates
 * per block: out[0] = gates of the first launch, out[1] = gates of the
 * second (0: none), out[2] = its shape, out[3] = its blocks.  CE_EINVAL for
 * a null out, n_jobs < 0, a shape outside 1-4 or blocks < 1. */
ce_status ce_blind_rotate_plan(int n_jobs, int gates_per_block, int blocks, int *out);
/* Engine of the fused sample extraction + key switching (§3: one key switch
 * per gate): 0 = automatic (tensor cores for single-client launches of at
 * least 32 outputs, CUDA cores otherwise), 1 = CUDA cores always, 2 = tensor
 * cores for every single-client launch.  On the tensor cores the key switch
 * is the exact product of a one-hot digit matrix and the key split into three
 * 11-bit fp16 limbs (fp32 sums of at most 8192 terms below 2^11 are exact);
 * both engines give bit-identical results.  CE_EINVAL for other values.
 * Applies to later calls. */
ce_status ce_set_keyswitch_config(ce_ctx *ctx, int engine);
/* Form of the external products inside blind rotation (§3: the CMux steps
 * of TFHE's bootstrapping): 0 = two-prime negacyclic transform on the CUDA
 * cores (default); 1 = Toeplitz form on the tensor cores, where each CMux
 * step of a batch is one [gates x 6144 digits] x [6144 x 2048] product with
 * the key's negacyclic Toeplitz blocks, key words split into four balanced
 * byte limbs and digits into two balanced 5-bit limbs (fp16 operands, fp32
 * sums of 6144 products of at most 2^11: exact integers), recombined mod
 * 2^32.  Both forms give bit-identical ciphertexts.  The tensor form applies
 * to single-client launches (batches, and engine levels of one client); it
 * builds the client's key as Hankel limb sequences (783,360,000 bytes,
 * counted against the HBM budget: CE_EADMIT if over it) on the first call
 * that uses it, so make that first call outside a stream capture.
 * CE_EINVAL for other values.  Applies to later calls. */
ce_status ce_set_external_product_form(ce_ctx *ctx, int form);
/* Failure-detection self-test (the paper has no counterpart to this call):
 * launches, on the context's stream, a kernel whose single thread waits on a
 * shared-memory barrier that nothing completes, using the library's bounded
 * device wait with limit_ns (1 us .. 2 s) instead of the kernels' 2 s.  The
 * wait expires and raises the context's device error flag, so the next
 * ce_synchronize returns CE_ETIMEOUT (and clears the flag); the context stays
 * usable.  CE_EINVAL for a limit outside the range. */
ce_status ce_selftest_device_wait(ce_ctx *ctx, uint64_t limit_ns);
/* Waits for the context's stream and reports a device-side failure of the
 * asynchronous calls since the previous check (CE_ETIMEOUT when a bounded
 * device wait expired). */
ce_status ce_synchronize(ce_ctx *ctx);
/* Project autotuner: times the blind-rotation kernel in each launch shape
 * (1, 2, 4 gates per block and the one-gate three-group shape) at a ladder of batch sizes (1 .. 9728 gates, synthetic inputs,
 * the client's key) and keeps the fastest shape per size; later launches
 * with the automatic shape use the nearest measured size.  Writes up to cap
 * (size, gates per block) pairs and their count.  Takes a few seconds. */
ce_status ce_autotune(ce_ctx *ctx, int client, int *out_jobs, int *out_g, int cap, int *count);
/* Number of kernels the last ce_gates_batch[_device] / ce_mux_batch_device
 * call launched (for launch accounting). */
int ce_last_launch_count(ce_ctx *ctx);

/* ------------------------------------------------------ functional units --- */

/* Functional units of the emulator (§5 "Data Processing Units", §6
 * "Conditional Flags") as netlists of bootstrapped gates.  Inputs: a[w]
 * then b[w] (bit 0 first); CSEL: rn[w], rm[w], N, Z, C, V.  Outputs: w bits;
 * CMP: N, Z, C, V of a - b; ADDS/SUBS: w bits then N, Z, C, V; SMULL/UMULL:
 * 2w bits.  cond (CSEL only): 0 EQ, 1 NE, 2 CS, 3 CC, 4 MI,
 * 5 PL, 6 VS, 7 VC, 8 HI, 9 LS, 10 GE, 11 LT, 12 GT, 13 LE. */
typedef enum {
    CE_U_ADD = 0,         /* Kogge-Stone parallel-prefix adder (§5 "Adder") */
    CE_U_ADD_RIPPLE = 1,  /* ripple-carry adder */
    CE_U_SUB = 2,         /* a + NOT b + 1 (§5 "Subtractor") */
    CE_U_AND = 3,         /* bitwise AND (§5 "Bitwise operations") */
    CE_U_ORR = 4,         /* bitwise OR */
    CE_U_LSL = 5,         /* a << (b mod w), barrel shifter of MUX stages (§5 "Shifter") */
    CE_U_MUL = 6,         /* (a * b) mod 2^w, array multiplier (§5 "Multiplier") */
    CE_U_UDIV = 7,        /* a / b (0 for b = 0), non-restoring (§5 "Divider") */
    CE_U_CMP = 8,         /* NZCV flags of a - b (§6 "Conditional Flags") */
    CE_U_CSEL = 9,        /* cond(NZCV) ? rn : rm */
    CE_U_LSR = 10,        /* a >> (b mod w), the LSL barrel on the bit-reversed operand
                             (§5 "Logic right shift/Arithmetic right shift") */
    CE_U_ASR = 11,        /* signed a >> (b mod w): as LSR, the MSB shifted in */
    CE_U_EOR = 12,        /* bitwise XOR (§5 "Bitwise operations") */
    CE_U_ORN = 13,        /* bitwise a OR NOT b */
    CE_U_ADDS = 14,       /* a + b then its N, Z, C, V (outputs w + 4) */
    CE_U_SUBS = 15,       /* a - b then its N, Z, C, V (CMP keeping the difference) */
    CE_U_SMULL = 16,      /* signed a * b, the full 2w-bit product, low half first
                             (§5 "Signed multiplication": carry-save array, sign
                             extension replaced by a constant; outputs 2w) */
    CE_U_UMULL = 17,      /* unsigned a * b, the full 2w-bit product (§5 "Unsigned
                             multiplication", as an array; outputs 2w) */
    CE_U_ADD_MUX = 18,    /* ADD's parallel-prefix adder (§5 "Adder") with each span
                             combine's carry as one MUX, G = P ? G' : G, instead of
                             AND then OR: the same bootstraps in fewer levels */
    CE_U_SUB_MUX = 19,    /* SUB (§5 "Subtractor") with that adder */
    CE_U_MUL_TREE = 20,   /* MUL's low half (§5 "Multiplier") by column compression: full
                             adders on three bits of a weight per stage (a Wallace
                             tree), then the MUX-carry adder; more bootstraps, fewer
                             levels than the array */
    CE_U_UDIV_MUX = 21    /* UDIV (§5 "Divider") with the MUX-carry adder in every
                             step (its encrypted carry-in folded in by a MUX too) */
} ce_unit;

/* Shape of a unit's netlist for width w (a power of two, 2..32). */
ce_status ce_unit_info(int unit, int cond, int width, int *n_inputs, int *n_outputs,
                       int *n_gates, int *n_bootstraps, int *depth);
/* The netlist as int32 words: n_inputs, n_wires, depth, n_gates, n_outputs;
 * per gate (ordered by level): op (0..9 gate, 10 MUX), a.wire, a.neg,
 * b.wire, b.neg, c.wire, c.neg (MUX selector a: a ? b : c), out, level; per
 * output: wire, neg.  Wire -1 is the constant false (negated: true).  With
 * buf NULL only *used is set. */
ce_status ce_unit_netlist(int unit, int cond, int width, int32_t *buf, size_t cap, size_t *used);

/* Evaluates a unit over n independent operand sets on device buffers:
 * d_in is [n][n_inputs][501] ciphertexts, d_out [n][n_outputs][501].  All
 * gates of one level of all n sets form one batched launch (linear
 * combination + modulus switch, blind rotation, extraction + key switch);
 * the whole unit is planned once per (unit, cond, n, buffers) and replayed
 * as a captured CUDA graph on `cuda_stream` (asynchronous). */
ce_status ce_unit_eval_device(ce_ctx *ctx, int client, int unit, int cond,
                              const uint32_t *d_in, uint32_t *d_out, size_t n,
                              void *cuda_stream);
/* The same at any width w (a power of two, 2..32; the paper's 32-bit units,
 * §5): d_in [n][2w (CSEL: 2w + 4)][501], d_out [n][w (CMP: 4)][501].
 * (SMULL/UMULL: [n][2w][501]).  ce_unit_eval_device is this call with width 16.  CE_EINVAL for another
 * width. */
ce_status ce_unit_eval_device_width(ce_ctx *ctx, int client, int unit, int cond, int width,
                                    const uint32_t *d_in, uint32_t *d_out, size_t n,
                                    void *cuda_stream);
/* The same with host buffers (blocking): in is [n][n_inputs] host
 * ciphertexts, out [n][n_outputs]; the call copies the inputs to
 * context-owned device buffers, replays the unit's plan (captured graph) on
 * the context's stream and copies the results back.  Use pinned host memory
 * for full copy bandwidth.  Errors as ce_unit_eval_device, plus CE_ETIMEOUT /
 * CE_EINVAL for a device-side failure of this call's work. */
ce_status ce_unit_eval(ce_ctx *ctx, int client, int unit, int cond, int width,
                       const ce_lwe *in, ce_lwe *out, size_t n);
/* Graph replay (1, default) or eager launches (0) for ce_unit_eval_device,
 * ce_unit_eval and register programs (ce_exec, ce_exec_multi): with graphs
 * on, a program set is planned on its first run (every tick recorded on the
 * host against slots the plan owns) and replayed as one captured CUDA graph,
 * the clients' registers copied in and out; results are bit-identical to
 * the eager tick loop.  Program calls with a host time limit (timeout_ns >
 * 0) always run the eager tick loop. */
ce_status ce_set_unit_graphs(ce_ctx *ctx, int on);
/* Level batching (1, default) or, for comparison, one launch per gate and
 * step (0): with batching off, every level of ce_unit_eval*, ce_exec* and
 * the server runs each gate as launches of its own (its linear combination,
 * its blind rotation in the one-gate shape, its extraction + key switch on
 * the CUDA cores) instead of one batched launch per step.  Results are
 * bit-identical; only the launch structure and the time change.  No paper
 * passage: a measurement mode that sets gate-at-a-time evaluation against
 * the level-batched engine. */
ce_status ce_set_level_batching(ce_ctx *ctx, int on);
/* Circuits of the instructions ADD, SUB, MUL and UDIV in ce_exec*,
 * ce_exec_branching and the server: 0 (default) the paper's (CE_U_ADD,
 * CE_U_SUB, CE_U_MUL, CE_U_UDIV), 1 the low-latency ones with the same
 * semantics (CE_U_ADD_MUX, CE_U_SUB_MUX, CE_U_MUL_TREE, CE_U_UDIV_MUX: fewer
 * levels, MUL_TREE with more bootstraps).  Applies to
 * instructions started later; register results decrypt to the same values,
 * their ciphertexts differ. */
ce_status ce_set_instruction_circuits(ce_ctx *ctx, int low_latency);

/* ------------------------------------------- encrypted register programs --- */

/* Instructions over a client's encrypted register file of 8 16-bit
 * registers and its encrypted NZCV flags (§4 "Data Processing": load-store
 * machine over vRegs; §6 conditional flags).  The program counter and the
 * instructions are cleartext; registers and flags stay encrypted. */
typedef enum {
    CE_I_ADD = 0,      /* rd = rn + rm (§5 "Adder": parallel-prefix adder) */
    CE_I_SUB = 1,      /* rd = rn - rm (§5 "Subtractor") */
    CE_I_AND = 2,      /* rd = rn & rm (§5 "Bitwise operations") */
    CE_I_ORR = 3,      /* rd = rn | rm (§5 "Bitwise operations") */
    CE_I_LSL = 4,      /* rd = rn << (rm mod 16) (§5 "Shifter": barrel shifter) */
    CE_I_LSL_IMM = 5,  /* rd = rn << (imm mod 16) (§5 "Shifter", shift immediate: no bootstrap) */
    CE_I_MUL = 6,      /* rd = (rn * rm) mod 2^16 (§5 "Multiplier") */
    CE_I_UDIV = 7,     /* rd = rn / rm, 0 when rm = 0 (§5 "Divider") */
    CE_I_CMP = 8,      /* NZCV = flags(rn - rm) (§6 "Conditional Flags") */
    CE_I_CSEL = 9,     /* rd = cond(NZCV) ? rn : rm (cond as for CE_U_CSEL; §6
                          conditional execution on the encrypted flags) */
    CE_I_MOV = 10,     /* rd = rn (§5 "Data movement": COPY, no bootstrap) */
    CE_I_MOV_IMM = 11, /* rd = imm (8-bit, zero extended; trivial ciphertexts:
                          §3 CONSTANT) */
    CE_I_LSR = 12,     /* rd = rn >> (rm mod 16), logical (§5 "Logic right
                          shift/Arithmetic right shift": barrel shifter) */
    CE_I_ASR = 13,     /* rd = rn >> (rm mod 16), arithmetic (same passage) */
    CE_I_LSR_IMM = 14, /* rd = rn >> (imm mod 16), logical (no bootstrap) */
    CE_I_ASR_IMM = 15, /* rd = rn >> (imm mod 16), arithmetic (no bootstrap) */
    CE_I_EOR = 16,     /* rd = rn ^ rm (§5 "Bitwise operations") */
    CE_I_ORN = 17,     /* rd = rn | ~rm (§5 "Bitwise operations") */
    /* §5 "Bitwise operations" with an immediate and NOT, and "Data movement":
     * no bootstrap (wire copies, negations and constants).  imm: 8 bits, zero
     * extended; BFC/BFI: field lsb = imm & 15, width = (imm >> 4) + 1, clipped
     * at bit 15. */
    CE_I_MVN = 18,     /* rd = ~rn */
    CE_I_AND_IMM = 19, /* rd = rn & imm */
    CE_I_ORR_IMM = 20, /* rd = rn | imm */
    CE_I_EOR_IMM = 21, /* rd = rn ^ imm */
    CE_I_BFC = 22,     /* clear bits [lsb, lsb + width) of rd */
    CE_I_BFI = 23,     /* rd[lsb, lsb + width) = rn[0, width) */
    CE_I_RBIT = 24,    /* rd = rn with the bit order reversed */
    CE_I_REV = 25,     /* rd = rn with the two bytes swapped */
    CE_I_ADDS = 26,    /* rd = rn + rm, NZCV = its flags (§6 "Conditional Flags":
                          the flag-setting form) */
    CE_I_SUBS = 27,    /* rd = rn - rm, NZCV = flags(rn - rm) (§6, the SUBS example) */
    CE_I_SMULH = 28,   /* rd = bits 16..31 of the signed product rn * rm (§5 "Signed
                          multiplication"; the low half is CE_I_MUL's) */
    CE_I_UMULH = 29,   /* rd = bits 16..31 of the unsigned product rn * rm */
    /* Branches (§6 "Branch"): the program counter is cleartext; only
     * ce_exec_branching runs them.  imm is the target instruction index
     * (equal to the program length: end the program). */
    CE_I_BCOND = 30,   /* if cond(NZCV) then pc = imm, decided by the key owner */
    CE_I_B = 31        /* pc = imm */
} ce_opcode;
/* One cleartext instruction (§4 "Cloud service model": HE instructions are
 * unencrypted; §4 "Data Processing": register operands rd, rn, rm are vReg
 * indices 0..7, imm an 8-bit immediate, cond a condition code as for
 * CE_U_CSEL). */
typedef struct { uint8_t op, rd, rn, rm, imm, cond; } ce_insn;

/* Register file access with host ciphertexts (bit 0 first; blocking): the
 * encrypted vRegs of §4 "Data Processing", which the user fills and reads
 * through the cloud service model (§4 "Cloud service model").  Registers
 * not written hold trivial encryptions of 0.  CE_EINVAL for reg outside
 * 0..7, CE_ENOTFOUND for an unknown client. */
ce_status ce_reg_write(ce_ctx *ctx, int client, int reg, const ce_lwe bits[16]);
ce_status ce_reg_read(ce_ctx *ctx, int client, int reg, ce_lwe bits[16]);
/* The encrypted NZCV flags (§6 "Conditional Flags"), N first. */
ce_status ce_flags_read(ce_ctx *ctx, int client, ce_lwe nzcv[4]);
/* Runs a program to completion on the client's registers (§4: the emulator
 * fetches cleartext instructions and runs them over encrypted vRegs; §6
 * "Branch and Control Flow" for the flags): blocking on the host until every
 * instruction is enqueued; results are read with ce_reg_read.  Malformed
 * instructions and branches (ce_exec_branching runs those) give CE_EINVAL;
 * timeout_ns > 0 bounds the host time (CE_ETIMEOUT). */
ce_status ce_exec(ce_ctx *ctx, int client, const ce_insn *prog, size_t n, uint64_t timeout_ns);
/* Branch resolution by the key owner (§6 "Branch": the cloud sends the
 * encrypted NZCV and the branch condition to a machine that owns the secret
 * key, which decrypts them and returns the decision).  Called on the thread
 * that runs ce_exec_branching, with no context lock held; nzcv (N first) is
 * valid during the call.  Returns 1 (taken), 0 (not taken) or a negative
 * value to abort the program. */
typedef int (*ce_branch_fn)(void *user, int client, uint8_t cond, const ce_lwe *nzcv);
/* Runs a program with branches (§6 "Branch and Control Flow": fetch at the
 * cleartext PC, execute over encrypted vRegs, B.cond resolved through
 * `decide`).  Straight-line runs between branches go through the engine as
 * in ce_exec.  At most 256 instructions; max_steps > 0 bounds the executed
 * instructions and timeout_ns > 0 the host time (CE_ETIMEOUT either way);
 * *steps_out (may be NULL) receives the executed count.  CE_EINVAL for a
 * target beyond the program end, a malformed instruction, or a negative
 * decision. */
ce_status ce_exec_branching(ce_ctx *ctx, int client, const ce_insn *prog, size_t n,
                            ce_branch_fn decide, void *user, uint64_t max_steps,
                            uint64_t timeout_ns, uint64_t *steps_out);
/* Runs several programs concurrently (§5: independent work of the emulator
 * runs in parallel; here across programs and clients): their instructions
 * advance level by level together, so gates of different programs and
 * clients share each batched launch. */
ce_status ce_exec_multi(ce_ctx *ctx, size_t n_programs, const int *clients,
                        const ce_insn *const *progs, const size_t *lens, uint64_t timeout_ns);

/* ---------------------------------------------------------------- serving --- */

/* A serving loop on a context (§4 "Cloud service model"): requests are single
 * instructions (ce_insn) on a client's encrypted registers, submitted from
 * any host thread.  A worker thread batches them continuously: each tick
 * starts queued requests (one in flight per client, so each client's
 * requests run in submission order, at most max_inflight in total; 0 = no
 * limit), runs one level of every in-flight instruction of every client in
 * one batched launch, and retires finished ones.  Requests arriving while
 * others run join at the next tick.  Results are bit-identical to running
 * the same instruction alone.  While a server runs, the context's other
 * calls take turns with its ticks (the context lock) and their GPU work is
 * ordered with the ticks' work. */
typedef struct ce_server ce_server;
ce_status ce_server_create(ce_ctx *ctx, int max_inflight, ce_server **out);
/* Enqueue one instruction (any ce_opcode) for `client`; *ticket identifies
 * the request.  CE_ENOTFOUND for an unknown client, CE_EINVAL for a
 * malformed instruction. */
ce_status ce_server_submit(ce_server *s, int client, const ce_insn *insn, uint64_t *ticket);
/* Non-blocking status; times are steady-clock nanoseconds (submission,
 * start on the GPU path, completion of its GPU work). */
ce_status ce_server_poll(ce_server *s, uint64_t ticket, int *done, uint64_t *submit_ns,
                         uint64_t *start_ns, uint64_t *done_ns);
/* Wait for a request (timeout_ns = 0: no limit; CE_ETIMEOUT on expiry). */
ce_status ce_server_wait(ce_server *s, uint64_t ticket, uint64_t timeout_ns);
ce_status ce_server_stats(ce_server *s, uint64_t *ticks, uint64_t *bootstraps,
                          uint64_t *queued, uint64_t *running);
/* Finishes every submitted request, then stops the worker. */
void ce_server_destroy(ce_server *s);

/* The paper has no counterpart to this call.  Same as ce_gates_batch_device
 * (same kernels, same results) but it allocates no device memory: for
 * callers that cannot let the library call cudaMalloc, e.g. a serving loop
 * that must not take cudaMalloc's implicit device-wide synchronisation, or a
 * process whose device memory another allocator has reserved up front.  Its
 * scratch is a fixed area inside the library's device image (about 2.3 MB
 * on every GPU that loads the library, held until the process exits), so a
 * call takes at most 256 gates (CE_EINVAL above that).  The first call on a
 * device looks up that area's address (cudaGetSymbolAddress); make that
 * first call before any stream capture.  Every call reuses the same area:
 * calls whose work overlaps on the GPU (different streams, different
 * contexts) race and corrupt each other's results, so serialise them.  No
 * scratch word needs to start at zero: each call writes everything it reads.
 * The keys are the client's keys held by the context (admitted earlier).
 * It always uses the transform form of the external products and the
 * CUDA-core key switch (whose scratch fits the fixed area).  Its launches
 * appear in ce_profile_read and ce_last_launch_count like the others. */
ce_status ce_gates_batch_device_noalloc(ce_ctx *ctx, int client, const uint8_t *d_ops,
                                        const uint32_t *d_a, const uint32_t *d_b,
                                        uint32_t *d_out, size_t n, void *cuda_stream);

/* ------------------------------------------------------------ gate trace --- */

/* One traced gate of the netlist engine (for verification; the paper has no
 * counterpart): the gate exactly as the GPU evaluated it, so that a plain
 * CPU implementation can recompute its output from the GPU's own inputs.
 * op: 0..9 a ce_gate_op on (in[0], in[1]); 10 MUX in[0] ? in[1] : in[2].
 * neg[i]: input i enters negated (the netlist's free NOT).  in[i] are the
 * words stored on the GPU before that negation (in[2] is zero unless MUX).
 * tick: the engine tick (one level of every in-flight instruction) counted
 * from ce_trace_enable; index: the gate's output position within its tick. */
typedef struct {
    int32_t op;
    int32_t neg[3];
    int32_t client;
    uint32_t tick;
    uint32_t index;
    uint32_t pad;
    ce_lwe in[3];
    ce_lwe out;
} ce_trace_rec;
/* Start (per_tick > 0) or stop (0) tracing: from now on every engine tick
 * (functional units, programs, serving) records up to per_tick of its gates,
 * spread evenly over the tick's outputs, into a context-owned device buffer
 * of cap records (each 8,048 bytes; records beyond cap are counted but not
 * kept).  Waits for all work on the device and clears earlier records.
 * While tracing, units run eagerly instead of as captured graphs (same
 * kernels, same results) plus one small copy kernel per tick.  CE_EINVAL for
 * per_tick above 4096 or cap outside 1..2^20 (when per_tick > 0). */
ce_status ce_trace_enable(ce_ctx *ctx, int per_tick, size_t cap);
/* Copies up to cap of the records kept since the last read into out (host
 * memory), in the order the GPU wrote them, and clears them: *count = records
 * copied, *seen (may be NULL) = records made, kept or not.  Waits for all
 * work on the device. */
ce_status ce_trace_read(ce_ctx *ctx, ce_trace_rec *out, size_t cap, size_t *count,
                        uint64_t *seen);

/* Measurement of the integer multiply-add pipe (the paper has no counterpart;
 * the blind rotation's binding unit): every SM runs chained operations of
 * three kinds — 32-bit multiply-add, high half of a 32 x 32-bit product, and
 * 32 x 32 -> 64-bit multiply-add — timed with the SM clock, and writes the
 * lane operations per clock per SM of each kind into lane_ops_per_clock[3].
 * Blocking; takes about a millisecond. */
ce_status ce_probe_int_pipes(ce_ctx *ctx, double *lane_ops_per_clock);

/* Per-kernel timing for measurement: while enabled, every kernel launch of
 * the gate path is bracketed by CUDA events on its own stream.
 * ce_profile_read waits for them and returns, per kernel kind (0 = linear
 * combination + modulus switch, 1 = blind rotation, 2 = extraction + key
 * switching, 3 = the MMA launches inside a tensor-core blind rotation, also
 * counted in kind 1), the summed milliseconds and the launch count since the
 * last read. */
ce_status ce_profile_enable(ce_ctx *ctx, int on);
ce_status ce_profile_read(ce_ctx *ctx, double *ms, int *launches, int kinds);

#ifdef __cplusplus
}
#endif
#endif
