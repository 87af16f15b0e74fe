/*
 * Plain CPU oracle for TFHE gate bootstrapping — TEST INFRASTRUCTURE ONLY.
 * See tfhe_oracle.h for scope.  Slow on purpose: every step is written the way
 * its definition reads, with no blocking, fusion or transform tricks.
 *
 * Sources for each step: the paper fixes the gate set and its truth tables
 * (§3, Table "TFHE API Benchmark") and that a binary gate costs one bootstrap
 * and MUX two (§3, text after the table).  The bootstrapping construction is
 * the TFHE one cited in §2/§3; the conventions it leaves open are stated at
 * each function.
 */
#include "tfhe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- PRNG --- */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the k-th output (k = 0, 1,
 * ...) of the generator seeded with `seed` is mix(seed + (k + 1) * gamma). */
uint64_t or_splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform uint32 number i of a domain: the high 32 bits of SplitMix64 output
 * domain * 2^40 + i.  Each domain owns a disjoint segment of one stream. */
uint32_t or_uniform32(uint64_t seed, uint32_t domain, uint64_t i)
{
    return (uint32_t)(or_splitmix64_at(seed, ((uint64_t)domain << 40) + i) >> 32);
}

/* Gaussian torus noise number i of a domain: Box-Muller on uniforms 2i and
 * 2i+1, u1 in (0,1], u2 in [0,1); z = sqrt(-2 ln u1) cos(2 pi u2); the noise
 * is round-to-nearest(sigma * 2^32 * z) taken mod 2^32. */
uint32_t or_gauss32(uint64_t seed, uint32_t domain, uint64_t i, double sigma)
{
    uint32_t x1 = or_uniform32(seed, domain, 2 * i);
    uint32_t x2 = or_uniform32(seed, domain, 2 * i + 1);
    double u1 = ((double)x1 + 1.0) / 4294967296.0;
    double u2 = (double)x2 / 4294967296.0;
    double z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    double e = (sigma * 4294967296.0) * z;
    return (uint32_t)(int64_t)llround(e);
}

/* -------------------------------------------------------- polynomials --- */

/* Schoolbook product in Z_{2^32}[X]/(X^N + 1): out_k = sum_{i+j=k} a_i b_j -
 * sum_{i+j=k+N} a_i b_j.  Accumulated in 64-bit wrapping integers, which is
 * exact mod 2^32. */
void or_poly_mul(int32_t N, const uint32_t *a, const uint32_t *b, uint32_t *out)
{
    uint64_t *acc = (uint64_t *)calloc((size_t)N, sizeof(uint64_t));
    for (int32_t i = 0; i < N; i++) {
        uint64_t ai = a[i];
        for (int32_t j = 0; j < N; j++) {
            int32_t k = i + j;
            if (k < N) acc[k] += ai * (uint64_t)b[j];
            else       acc[k - N] -= ai * (uint64_t)b[j];
        }
    }
    for (int32_t k = 0; k < N; k++) out[k] = (uint32_t)acc[k];
    free(acc);
}

/* out += d * b for a signed digit polynomial d, in signed 64-bit integers
 * (|d_i| <= Bg/2, b_j < 2^32: every partial sum stays far below 2^63). */
static void poly_muladd_digit(int32_t N, const int32_t *d, const uint32_t *b,
                              int64_t *out)
{
    for (int32_t i = 0; i < N; i++) {
        int64_t di = d[i];
        if (di == 0) continue;
        for (int32_t j = 0; j < N; j++) {
            int32_t k = i + j;
            if (k < N) out[k] += di * (int64_t)b[j];
            else       out[k - N] -= di * (int64_t)b[j];
        }
    }
}

/* X^k * p for k in [0, 2N): coefficient j is p_{j-k} if j >= k, else
 * -p_{j-k+N} (for k < N); X^N = -1 handles k >= N. */
static void poly_rotate(int32_t N, const uint32_t *p, int32_t k, uint32_t *out)
{
    int32_t neg = 0;
    k %= 2 * N;
    if (k < 0) k += 2 * N;
    if (k >= N) { k -= N; neg = 1; }
    for (int32_t j = 0; j < N; j++) {
        uint32_t v = (j >= k) ? p[j - k] : (uint32_t)(0u - p[j - k + N]);
        out[j] = neg ? (uint32_t)(0u - v) : v;
    }
}

/* ------------------------------------------------------------- keygen --- */

/* Secret keys: LWE key s in {0,1}^n and TRLWE key K in B[X]/(X^N+1), each bit
 * the top bit of one uniform draw. */
void or_secret_keygen(const or_params *p, uint64_t seed, uint32_t *s, uint32_t *K)
{
    for (int32_t i = 0; i < p->n; i++) s[i] = or_uniform32(seed, OR_DOM_LWE_KEY, i) >> 31;
    for (int32_t j = 0; j < p->N; j++) K[j] = or_uniform32(seed, OR_DOM_TRLWE_KEY, j) >> 31;
}

/* Bootstrapping key: for each LWE key bit s_i a TRGSW encryption of s_i under
 * K, stored as 2l TRLWE rows of two polynomials (a, b).  Row r = c*l + (p-1)
 * (c = 0: a-part, c = 1: b-part, p = 1..l) is a TRLWE encryption of zero,
 * b = a*K + e, with s_i * 2^(32 - Bgbit*p) added to the constant coefficient of
 * component c.  Layout: bsk[((i*2l + r)*2 + comp)*N + j]. */
void or_bsk_keygen(const or_params *p, uint64_t seed, const uint32_t *s,
                   const uint32_t *K, uint32_t *bsk)
{
    const int32_t N = p->N, rows = 2 * p->l;
    uint32_t *aK = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)N);
    for (int32_t i = 0; i < p->n; i++) {
        for (int32_t r = 0; r < rows; r++) {
            uint64_t base = ((uint64_t)i * rows + r) * (uint64_t)N;
            uint32_t *ra = bsk + (base * 2);
            uint32_t *rb = ra + N;
            for (int32_t j = 0; j < N; j++) ra[j] = or_uniform32(seed, OR_DOM_BSK_A, base + j);
            or_poly_mul(N, ra, K, aK);
            for (int32_t j = 0; j < N; j++)
                rb[j] = aK[j] + or_gauss32(seed, OR_DOM_BSK_E, base + j, p->sigma_bk);
            int32_t c = r / p->l, pp = r % p->l + 1;
            uint32_t h = (uint32_t)1u << (32 - p->Bgbit * pp);
            if (c == 0) ra[0] += s[i] * h;
            else        rb[0] += s[i] * h;
        }
    }
    free(aK);
}

/* Key-switching key: KSK[j][q][v] = LWE_s(v * K_j * 2^(32 - basebit*(q+1)))
 * for j < N, q < t, v < 2^basebit (v = 0 rows are stored and never used).
 * Layout: ksk[(((j*t + q)*B + v)*(n+1)) + m], m = n is the b word. */
void or_ksk_keygen(const or_params *p, uint64_t seed, const uint32_t *s,
                   const uint32_t *K, uint32_t *ksk)
{
    const int32_t n = p->n, B = 1 << p->basebit;
    for (int32_t j = 0; j < p->N; j++)
        for (int32_t q = 0; q < p->t; q++)
            for (int32_t v = 0; v < B; v++) {
                uint64_t idx = ((uint64_t)j * p->t + q) * B + v;
                uint32_t *row = ksk + idx * (uint64_t)(n + 1);
                uint32_t b = 0;
                for (int32_t m = 0; m < n; m++) {
                    row[m] = or_uniform32(seed, OR_DOM_KSK_A, idx * (uint64_t)n + m);
                    b += row[m] * s[m];
                }
                uint32_t msg = (uint32_t)v * K[j] * ((uint32_t)1u << (32 - p->basebit * (q + 1)));
                row[n] = b + or_gauss32(seed, OR_DOM_KSK_E, idx, p->sigma_lwe) + msg;
            }
}

/* ------------------------------------------------------- enc / dec --- */

#define MU_EIGHTH 0x20000000u  /* +1/8 on the torus */

/* LWE encryption of a bit: a uniform, b = <a,s> + e + (bit ? +1/8 : -1/8). */
void or_encrypt(const or_params *p, const uint32_t *s, int bit, uint64_t seed,
                uint64_t ctr, uint32_t *out)
{
    uint32_t b = 0;
    for (int32_t m = 0; m < p->n; m++) {
        out[m] = or_uniform32(seed, OR_DOM_ENC_A, ctr * (uint64_t)p->n + m);
        b += out[m] * s[m];
    }
    b += or_gauss32(seed, OR_DOM_ENC_E, ctr, p->sigma_lwe);
    b += bit ? MU_EIGHTH : (uint32_t)(0u - MU_EIGHTH);
    out[p->n] = b;
}

/* Phase b - <a,s> mod 2^32. */
uint32_t or_phase(const or_params *p, const uint32_t *s, const uint32_t *c)
{
    uint32_t ph = c[p->n];
    for (int32_t m = 0; m < p->n; m++) ph -= c[m] * s[m];
    return ph;
}

/* Decryption: the bit is 1 iff the phase, read as a signed torus value, is
 * positive. */
int or_decrypt(const or_params *p, const uint32_t *s, const uint32_t *c)
{
    return (int32_t)or_phase(p, s, c) > 0;
}

/* --------------------------------------------------- gadget / modswitch --- */

/* Balanced gadget decomposition: x is first rounded to the nearest multiple
 * of 2^(32 - l*Bgbit) (ties up); the digits d_1..d_l in [-Bg/2, Bg/2) are the
 * unique ones with sum_p d_p 2^(32 - Bgbit*p) equal to the rounded x mod 2^32.
 * They are read off x + round-offset + sum_p (Bg/2) 2^(32 - Bgbit*p). */
void or_decompose(const or_params *p, uint32_t x, int32_t *digits)
{
    const int32_t Bgbit = p->Bgbit, l = p->l;
    const uint32_t half = 1u << (Bgbit - 1), mask = (1u << Bgbit) - 1;
    uint32_t w = x;
    int32_t dropped = 32 - l * Bgbit;
    if (dropped > 0) w += 1u << (dropped - 1);
    for (int32_t pp = 1; pp <= l; pp++) w += half << (32 - Bgbit * pp);
    for (int32_t pp = 1; pp <= l; pp++)
        digits[pp - 1] = (int32_t)((w >> (32 - Bgbit * pp)) & mask) - (int32_t)half;
}

/* Modulus switch from 2^32 to 2N: round(x * 2N / 2^32) mod 2N, ties up. */
uint32_t or_modswitch(uint32_t x, int32_t N)
{
    int32_t sh = 32;
    for (int32_t m = 2 * N; m > 1; m >>= 1) sh--;   /* sh = 32 - log2(2N) */
    return ((x + (1u << (sh - 1))) >> sh) & (uint32_t)(2 * N - 1);
}

/* ------------------------------------------------------------- gates --- */

/* Linear part of each bootstrapped gate: (0, kappa) + s1*c1 + s2*c2, with
 * kappa in eighths of the torus.  With bits encoded as +-1/8 the result's
 * phase is positive exactly on the gate's true rows (truth tables: §3, Table
 * "TFHE API Benchmark"; these are the TFHE gate formulas). */
static const int32_t GATE_KAPPA8[OR_NUM_GATES] = { 1, -1, 1, 2, -1, -2, -1, -1, 1, 1 };
static const int32_t GATE_S1[OR_NUM_GATES]     = { -1, 1, 1, 2, -1, -2, -1, 1, -1, 1 };
static const int32_t GATE_S2[OR_NUM_GATES]     = { -1, 1, 1, 2, -1, -2, 1, -1, 1, -1 };

void or_gate_lincomb(const or_params *p, int op, const uint32_t *c1,
                     const uint32_t *c2, uint32_t *out)
{
    uint32_t s1 = (uint32_t)GATE_S1[op], s2 = (uint32_t)GATE_S2[op];
    for (int32_t m = 0; m <= p->n; m++) out[m] = s1 * c1[m] + s2 * c2[m];
    out[p->n] += (uint32_t)GATE_KAPPA8[op] * MU_EIGHTH;
}

/* Blind rotation.  ACC starts as the trivial TRLWE (0, X^(-bbar) v) with the
 * test vector v = mu * sum_j X^j.  Step i (i = 0..n-1) is a CMux controlled by
 * s_i: D = X^(abar_i) ACC - ACC; each of D's two polynomials is split into l
 * digit polynomials; ACC += sum_r digit_r * BSK_i[r].  The result encrypts
 * X^(-bbar + sum abar_i s_i) v.  A step with abar_i = 0 has D = 0 and leaves
 * ACC unchanged.  acc layout: [comp a | comp b], N words each. */
void or_blind_rotate(const or_params *p, const uint32_t *bsk,
                     const uint32_t *abar, uint32_t bbar, uint32_t mu,
                     uint32_t *acc)
{
    const int32_t N = p->N, l = p->l, rows = 2 * l;
    uint32_t *v = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *rot = (uint32_t *)malloc(sizeof(uint32_t) * N);
    int32_t *dig = (int32_t *)malloc(sizeof(int32_t) * (size_t)rows * N);
    int64_t *sum = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)N);
    int32_t tmp[16];

    for (int32_t j = 0; j < N; j++) v[j] = mu;
    memset(acc, 0, sizeof(uint32_t) * N);
    poly_rotate(N, v, 2 * N - (int32_t)bbar, acc + N);

    for (int32_t i = 0; i < p->n; i++) {
        if (abar[i] == 0) continue;
        for (int32_t c = 0; c < 2; c++) {
            poly_rotate(N, acc + c * N, (int32_t)abar[i], rot);
            for (int32_t j = 0; j < N; j++) {
                or_decompose(p, rot[j] - acc[c * N + j], tmp);
                for (int32_t pp = 0; pp < l; pp++) dig[(c * l + pp) * N + j] = tmp[pp];
            }
        }
        memset(sum, 0, sizeof(int64_t) * 2 * N);
        for (int32_t r = 0; r < rows; r++) {
            const uint32_t *row = bsk + ((size_t)i * rows + r) * 2 * N;
            poly_muladd_digit(N, dig + r * N, row, sum);          /* a-part */
            poly_muladd_digit(N, dig + r * N, row + N, sum + N);  /* b-part */
        }
        for (int32_t j = 0; j < 2 * N; j++) acc[j] += (uint32_t)(uint64_t)sum[j];
    }
    free(v); free(rot); free(dig); free(sum);
}

/* Sample extraction of coefficient 0: the LWE sample under key K (as a vector
 * of N bits) with a'_0 = A_0, a'_j = -A_{N-j}, b' = B_0.  big has N+1 words. */
void or_sample_extract(const or_params *p, const uint32_t *acc, uint32_t *big)
{
    const int32_t N = p->N;
    big[0] = acc[0];
    for (int32_t j = 1; j < N; j++) big[j] = 0u - acc[N - j];
    big[N] = acc[N];
}

/* Key switching from dimension N (key K) to dimension n (key s): each a'_j is
 * rounded to t*basebit bits (ties up), split MSB-first into t unsigned base-B
 * digits, and out = (0, b') - sum_{j,q} KSK[j][q][digit_jq] (digit 0 adds
 * nothing). */
void or_key_switch(const or_params *p, const uint32_t *ksk, const uint32_t *big,
                   uint32_t *out)
{
    const int32_t n = p->n, N = p->N, t = p->t, bb = p->basebit, B = 1 << bb;
    const int32_t prec = t * bb;
    const uint32_t round = prec < 32 ? (1u << (31 - prec)) : 0u;
    for (int32_t m = 0; m < n; m++) out[m] = 0;
    out[n] = big[N];
    for (int32_t j = 0; j < N; j++) {
        uint32_t aj = big[j] + round;
        for (int32_t q = 0; q < t; q++) {
            uint32_t d = (aj >> (32 - bb * (q + 1))) & (uint32_t)(B - 1);
            if (d == 0) continue;
            const uint32_t *row = ksk + (((uint64_t)j * t + q) * B + d) * (uint64_t)(n + 1);
            for (int32_t m = 0; m <= n; m++) out[m] -= row[m];
        }
    }
}

/* Modulus switch of every word of an LWE sample (dimension n). */
static void modswitch_all(const or_params *p, const uint32_t *c, uint32_t *abar,
                          uint32_t *bbar)
{
    for (int32_t m = 0; m < p->n; m++) abar[m] = or_modswitch(c[m], p->N);
    *bbar = or_modswitch(c[p->n], p->N);
}

/* Bootstrap without key switching: modulus switch, blind rotation with test
 * vector +1/8, sample extraction (result of dimension N). */
static void bootstrap_no_ks(const or_params *p, const uint32_t *bsk,
                            const uint32_t *in, uint32_t *big)
{
    uint32_t *abar = (uint32_t *)malloc(sizeof(uint32_t) * p->n);
    uint32_t *acc = (uint32_t *)malloc(sizeof(uint32_t) * 2 * p->N);
    uint32_t bbar;
    modswitch_all(p, in, abar, &bbar);
    or_blind_rotate(p, bsk, abar, bbar, MU_EIGHTH, acc);
    or_sample_extract(p, acc, big);
    free(abar); free(acc);
}

void or_bootstrap(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                  const uint32_t *in, uint32_t *out)
{
    uint32_t *big = (uint32_t *)malloc(sizeof(uint32_t) * (p->N + 1));
    bootstrap_no_ks(p, bsk, in, big);
    or_key_switch(p, ksk, big, out);
    free(big);
}

void or_gate(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
             int op, const uint32_t *c1, const uint32_t *c2, uint32_t *out)
{
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (p->n + 1));
    or_gate_lincomb(p, op, c1, c2, lin);
    or_bootstrap(p, bsk, ksk, lin, out);
    free(lin);
}

/* MUX(a, b, c) = a ? b : c with two bootstraps and one key switch (§3: MUX is
 * bootstrapped twice): u1 = BR(AND-comb(a,b)), u2 = BR(ANDNY-comb(a,c)) in
 * dimension N, then KS((0, +1/8) + u1 + u2). */
void or_mux(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
            const uint32_t *a, const uint32_t *b, const uint32_t *c,
            uint32_t *out)
{
    const int32_t n = p->n, N = p->N;
    uint32_t *lin = (uint32_t *)malloc(sizeof(uint32_t) * (n + 1));
    uint32_t *u1 = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
    uint32_t *u2 = (uint32_t *)malloc(sizeof(uint32_t) * (N + 1));
    or_gate_lincomb(p, OR_AND, a, b, lin);
    bootstrap_no_ks(p, bsk, lin, u1);
    or_gate_lincomb(p, OR_ANDNY, a, c, lin);
    bootstrap_no_ks(p, bsk, lin, u2);
    for (int32_t j = 0; j <= N; j++) u1[j] += u2[j];
    u1[N] += MU_EIGHTH;
    or_key_switch(p, ksk, u1, out);
    free(lin); free(u1); free(u2);
}

/* Non-bootstrapped operations (§3, Table "TFHE API Benchmark"): CONSTANT is
 * the trivial sample (0, +-1/8); NOT negates every word. */
void or_constant(const or_params *p, int bit, uint32_t *out)
{
    for (int32_t m = 0; m < p->n; m++) out[m] = 0;
    out[p->n] = bit ? MU_EIGHTH : (uint32_t)(0u - MU_EIGHTH);
}

void or_not(const or_params *p, const uint32_t *c, uint32_t *out)
{
    for (int32_t m = 0; m <= p->n; m++) out[m] = 0u - c[m];
}

/* --------------------------------------------------------- batch helper --- */

/* Runs `count` independent gates on `threads` POSIX threads (gate g takes
 * ops[g], c1 + g*(n+1), c2 + g*(n+1) and writes out + g*(n+1)).  Each gate is
 * the plain or_gate above; threading only spreads independent gates over
 * cores for timing and large test batches. */
#include <pthread.h>

typedef struct {
    const or_params *p; const uint32_t *bsk, *ksk; const int32_t *ops;
    const uint32_t *c1, *c2; uint32_t *out; int64_t count; int64_t next;
    pthread_mutex_t lock;
} gate_job;

static void *gate_worker(void *arg)
{
    gate_job *jb = (gate_job *)arg;
    const int64_t w = jb->p->n + 1;
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int64_t g = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (g >= jb->count) break;
        or_gate(jb->p, jb->bsk, jb->ksk, jb->ops[g], jb->c1 + g * w, jb->c2 + g * w,
                jb->out + g * w);
    }
    return 0;
}

void or_gates_threaded(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                       const int32_t *ops, const uint32_t *c1, const uint32_t *c2,
                       uint32_t *out, int64_t count, int32_t threads)
{
    gate_job jb = { p, bsk, ksk, ops, c1, c2, out, count, 0, PTHREAD_MUTEX_INITIALIZER };
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int32_t i = 0; i < threads; i++) pthread_create(&th[i], 0, gate_worker, &jb);
    for (int32_t i = 0; i < threads; i++) pthread_join(th[i], 0);
    free(th);
}

/* Runs `count` independent MUX gates on `threads` POSIX threads (same plain
 * or_mux; threading only spreads independent gates over cores). */
typedef struct {
    const or_params *p; const uint32_t *bsk, *ksk;
    const uint32_t *a, *b, *c; uint32_t *out; int64_t count; int64_t next;
    pthread_mutex_t lock;
} mux_job;

static void *mux_worker(void *arg)
{
    mux_job *jb = (mux_job *)arg;
    const int64_t w = jb->p->n + 1;
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int64_t g = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (g >= jb->count) break;
        or_mux(jb->p, jb->bsk, jb->ksk, jb->a + g * w, jb->b + g * w, jb->c + g * w,
               jb->out + g * w);
    }
    return 0;
}

void or_muxes_threaded(const or_params *p, const uint32_t *bsk, const uint32_t *ksk,
                       const uint32_t *a, const uint32_t *b, const uint32_t *c,
                       uint32_t *out, int64_t count, int32_t threads)
{
    mux_job jb = { p, bsk, ksk, a, b, c, out, count, 0, PTHREAD_MUTEX_INITIALIZER };
    if (threads < 1) threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int32_t i = 0; i < threads; i++) pthread_create(&th[i], 0, mux_worker, &jb);
    for (int32_t i = 0; i < threads; i++) pthread_join(th[i], 0);
    free(th);
}
