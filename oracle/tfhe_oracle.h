/*
 * Plain CPU oracle for TFHE gate bootstrapping — TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline leg may load this code.  The product path (the CUDA library) never
 * includes, links or calls it, and shares no code with it.
 *
 * What it computes: the bootstrapped binary gates of the paper's §3 ("TFHE
 * Library", Table "TFHE API Benchmark"): a linear combination of two LWE
 * ciphertexts, the modulus switch to 2N, blind rotation (n CMux steps, each an
 * external product of a TRGSW bootstrapping-key row with the gadget-decomposed
 * TRLWE accumulator), sample extraction and LWE key switching.  The paper uses
 * TFHE as a black box (§3: one bootstrap per binary gate, two for MUX); the
 * construction is the one of the TFHE papers it cites in §2 and §3.  Every
 * convention the paper leaves open is written out next to the function that
 * uses it.  All arithmetic is exact integer arithmetic on the torus
 * T = R/Z represented as uint32 (x <-> x / 2^32); polynomial products are
 * schoolbook in 64-bit integers, reduced mod 2^32 and mod X^N + 1.
 *
 * All parameters are runtime values so that tests can run the same code at
 * tiny sizes; the gate workload uses n=500, N=1024, l=3, Bg=2^10, t=8,
 * base 2^2, sigma_lwe=2^-15, sigma_bk=9e-9.
 */
#ifndef TFHE_ORACLE_H
#define TFHE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n;          /* LWE dimension */
    int32_t N;          /* ring degree, power of two */
    int32_t l;          /* gadget length of the bootstrapping key */
    int32_t Bgbit;      /* log2 of the gadget base */
    int32_t t;          /* key-switch digit count */
    int32_t basebit;    /* log2 of the key-switch base */
    double sigma_lwe;   /* LWE / key-switching-key noise std (torus units) */
    double sigma_bk;    /* bootstrapping-key noise std (torus units) */
} or_params;

/* Gate opcodes (truth tables: §3, Table "TFHE API Benchmark"). */
enum { OR_NAND = 0, OR_AND, OR_OR, OR_XOR, OR_NOR, OR_XNOR,
       OR_ANDNY, OR_ANDYN, OR_ORNY, OR_ORYN, OR_NUM_GATES };

/* PRNG domains (one disjoint SplitMix64 stream segment per use). */
enum { OR_DOM_LWE_KEY = 1, OR_DOM_TRLWE_KEY = 2, OR_DOM_BSK_A = 3,
       OR_DOM_BSK_E = 4, OR_DOM_KSK_A = 5, OR_DOM_KSK_E = 6,
       OR_DOM_ENC_A = 7, OR_DOM_ENC_E = 8 };

uint64_t or_splitmix64_at(uint64_t seed, uint64_t k);
uint32_t or_uniform32(uint64_t seed, uint32_t domain, uint64_t i);
uint32_t or_gauss32(uint64_t seed, uint32_t domain, uint64_t i, double sigma);

void or_secret_keygen(const or_params *p, uint64_t seed, uint32_t *s, uint32_t *K);
void or_bsk_keygen(const or_params *p, uint64_t seed, const uint32_t *s,
                   const uint32_t *K, uint32_t *bsk);
void or_ksk_keygen(const or_params *p, uint64_t seed, const uint32_t *s,
                   const uint32_t *K, uint32_t *ksk);

void or_encrypt(const or_params *p, const uint32_t *s, int bit, uint64_t seed,
                uint64_t ctr, uint32_t *out);
uint32_t or_phase(const or_params *p, const uint32_t *s, const uint32_t *c);
int or_decrypt(const or_params *p, const uint32_t *s, const uint32_t *c);

void or_poly_mul(int32_t N, const uint32_t *a, const uint32_t *b, uint32_t *out);
void or_decompose(const or_params *p, uint32_t x, int32_t *digits);
uint32_t or_modswitch(uint32_t x, int32_t N);

void or_gate_lincomb(const or_params *p, int op, const uint32_t *c1,
                     const uint32_t *c2, uint32_t *out);
void or_blind_rotate(const or_params *p, const uint32_t *bsk,
                     const uint32_t *abar, uint32_t bbar, uint32_t mu,
                     uint32_t *acc);
void or_sample_extract(const or_params *p, const uint32_t *acc, uint32_t *big);
void or_key_switch(const or_params *p, const uint32_t *ksk, const uint32_t *big,
                   uint32_t *out);
void or_bootstrap(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                  const uint32_t *in, uint32_t *out);
void or_gate(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
             int op, const uint32_t *c1, const uint32_t *c2, uint32_t *out);
void or_mux(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
            const uint32_t *a, const uint32_t *b, const uint32_t *c,
            uint32_t *out);
void or_constant(const or_params *p, int bit, uint32_t *out);
void or_gates_threaded(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                       const int32_t *ops, const uint32_t *c1, const uint32_t *c2,
                       uint32_t *out, int64_t count, int32_t threads);
void or_not(const or_params *p, const uint32_t *c, uint32_t *out);
void or_muxes_threaded(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                       const uint32_t *a, const uint32_t *b, const uint32_t *c,
                       uint32_t *out, int64_t count, int32_t threads);

#ifdef __cplusplus
}
#endif
#endif
