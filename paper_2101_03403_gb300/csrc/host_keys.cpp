// Client-side key generation, encryption and decryption (host code of the
// library).  The paper's cloud service model (§4, "Cloud service model"): the
// client owns the secret key and hands the cloud key to the server; the
// TFHE API it uses offers secret/cloud keyset generation and bit
// encryption/decryption (§3, Table "TFHE API Benchmark").
//
// Randomness is counter based so that any key word can be regenerated
// independently: uniform draw i of domain d is the high 32 bits of output
// number d * 2^40 + i of SplitMix64 (Steele, Lea, Flood 2014) seeded with
// the caller's seed.  Gaussian noise i of a domain uses uniform draws 2i and
// 2i+1 through the Box-Muller transform.
#include "ce_internal.h"

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <thread>
#include <vector>

namespace ce {

namespace {

constexpr uint32_t kSecretMagic = 0x4B534543u;  // "CESK"
constexpr uint32_t kCloudMagic = 0x4B434543u;   // "CECK"
constexpr uint32_t kVersion = 1u;

enum Domain : uint32_t {
  kDomLweKey = 1, kDomRingKey = 2, kDomBskA = 3, kDomBskNoise = 4,
  kDomKskA = 5, kDomKskNoise = 6, kDomEncA = 7, kDomEncNoise = 8
};

inline uint64_t splitmix_output(uint64_t seed, uint64_t index) {
  // SplitMix64: state advances by the golden-ratio increment, then mixes.
  uint64_t x = seed + 0x9E3779B97F4A7C15ull * (index + 1ull);
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ull;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBull;
  x ^= x >> 31;
  return x;
}

inline uint32_t draw_u32(uint64_t seed, uint32_t dom, uint64_t i) {
  return static_cast<uint32_t>(splitmix_output(seed, (uint64_t(dom) << 40) + i) >> 32);
}

// Box-Muller: u1 in (0, 1], u2 in [0, 1), z = sqrt(-2 ln u1) cos(2 pi u2);
// the torus noise is sigma * 2^32 * z rounded to the nearest integer.
inline uint32_t draw_noise(uint64_t seed, uint32_t dom, uint64_t i, double sigma) {
  const double two32 = 4294967296.0;
  const double u1 = (static_cast<double>(draw_u32(seed, dom, 2 * i)) + 1.0) / two32;
  const double u2 = static_cast<double>(draw_u32(seed, dom, 2 * i + 1)) / two32;
  const double radius = std::sqrt(-2.0 * std::log(u1));
  const double z = radius * std::cos(2.0 * M_PI * u2);
  const double scaled = (sigma * two32) * z;
  return static_cast<uint32_t>(static_cast<int64_t>(std::llround(scaled)));
}

struct SecretView {
  const uint32_t *s;   // [kLweN]
  const uint32_t *K;   // [kRingN]
};

bool view_secret(const void *secret, SecretView *v) {
  if (!secret) return false;
  const uint32_t *w = static_cast<const uint32_t *>(secret);
  if (w[0] != kSecretMagic || w[1] != kVersion) return false;
  v->s = w + 2;
  v->K = w + 2 + kLweN;
  return true;
}

// TRLWE encryption of zero under binary key K: a uniform, b = a*K + e, with
// the product in Z_{2^32}[X]/(X^N+1) computed as a signed sum of rotations of
// a (K has 0/1 coefficients).
void trlwe_zero(uint64_t seed, uint64_t row, const uint32_t *K, uint32_t *a, uint32_t *b) {
  const uint64_t base = row * kRingN;
  for (int j = 0; j < kRingN; ++j) a[j] = draw_u32(seed, kDomBskA, base + j);
  for (int j = 0; j < kRingN; ++j) b[j] = draw_noise(seed, kDomBskNoise, base + j, kSigmaBsk);
  for (int k = 0; k < kRingN; ++k) {
    if (!K[k]) continue;
    // X^k * a: coefficient j is a[j-k] for j >= k and -a[j-k+N] below.
    for (int j = 0; j < k; ++j) b[j] -= a[j - k + kRingN];
    for (int j = k; j < kRingN; ++j) b[j] += a[j - k];
  }
}

}  // namespace

}  // namespace ce

using namespace ce;

extern "C" ce_status ce_secret_keygen(uint64_t seed, void **secret_out, size_t *bytes_out) {
  if (!secret_out) return set_error(CE_EINVAL, "ce_secret_keygen: null output");
  uint32_t *w = static_cast<uint32_t *>(std::malloc(CE_SECRET_BYTES));
  if (!w) return set_error(CE_ENOMEM, "ce_secret_keygen: out of host memory");
  w[0] = kSecretMagic;
  w[1] = kVersion;
  for (int i = 0; i < kLweN; ++i) w[2 + i] = draw_u32(seed, kDomLweKey, i) >> 31;
  for (int j = 0; j < kRingN; ++j) w[2 + kLweN + j] = draw_u32(seed, kDomRingKey, j) >> 31;
  *secret_out = w;
  if (bytes_out) *bytes_out = CE_SECRET_BYTES;
  return CE_OK;
}

extern "C" ce_status ce_cloud_keygen(const void *secret, uint64_t seed, void **cloud_out,
                                     size_t *bytes_out) {
  SecretView sk;
  if (!cloud_out || !view_secret(secret, &sk))
    return set_error(CE_EINVAL, "ce_cloud_keygen: bad secret key or null output");
  uint32_t *w = static_cast<uint32_t *>(std::malloc(CE_CLOUD_BYTES));
  if (!w) return set_error(CE_ENOMEM, "ce_cloud_keygen: out of host memory");
  w[0] = kCloudMagic;
  w[1] = kVersion;
  uint32_t *bsk = w + 2;
  uint32_t *ksk = bsk + CE_BSK_WORDS;

  unsigned nthreads = std::thread::hardware_concurrency();
  if (nthreads == 0) nthreads = 1;
  if (nthreads > 64) nthreads = 64;

  // Bootstrapping key: key bit i, row r = c*3 + (p-1): TRLWE_K(0) with
  // s_i * 2^(32 - 10p) added to the constant coefficient of component c.
  auto bsk_worker = [&](unsigned tid) {
    for (int i = static_cast<int>(tid); i < kLweN; i += static_cast<int>(nthreads)) {
      for (int r = 0; r < 2 * kGadgetL; ++r) {
        const uint64_t row = uint64_t(i) * (2 * kGadgetL) + r;
        uint32_t *a = bsk + row * 2 * kRingN;
        uint32_t *b = a + kRingN;
        trlwe_zero(seed, row, sk.K, a, b);
        const int c = r / kGadgetL, level = r % kGadgetL + 1;
        const uint32_t g = sk.s[i] << (32 - kBgBit * level);
        (c == 0 ? a : b)[0] += g;
      }
    }
  };
  // Key-switching key: LWE_s(v * K_j * 2^(32 - 2(q+1))), v = 0..3.
  auto ksk_worker = [&](unsigned tid) {
    for (int j = static_cast<int>(tid); j < kRingN; j += static_cast<int>(nthreads)) {
      for (int q = 0; q < kKsT; ++q) {
        for (int v = 0; v < kKsBase; ++v) {
          const uint64_t idx = (uint64_t(j) * kKsT + q) * kKsBase + v;
          uint32_t *row = ksk + idx * kLweWords;
          uint32_t acc = 0;
          for (int m = 0; m < kLweN; ++m) {
            row[m] = draw_u32(seed, kDomKskA, idx * kLweN + m);
            acc += row[m] * sk.s[m];
          }
          const uint32_t msg = uint32_t(v) * sk.K[j] * (1u << (32 - kKsBaseBit * (q + 1)));
          row[kLweN] = acc + draw_noise(seed, kDomKskNoise, idx, kSigmaLwe) + msg;
        }
      }
    }
  };
  std::vector<std::thread> pool;
  for (unsigned t = 0; t < nthreads; ++t) pool.emplace_back(bsk_worker, t);
  for (auto &th : pool) th.join();
  pool.clear();
  for (unsigned t = 0; t < nthreads; ++t) pool.emplace_back(ksk_worker, t);
  for (auto &th : pool) th.join();

  *cloud_out = w;
  if (bytes_out) *bytes_out = CE_CLOUD_BYTES;
  return CE_OK;
}

extern "C" void ce_free(void *p) { std::free(p); }

extern "C" ce_status ce_encrypt_bit(const void *secret, int bit, uint64_t seed, uint64_t ctr,
                                    ce_lwe *out) {
  SecretView sk;
  if (!out || !view_secret(secret, &sk))
    return set_error(CE_EINVAL, "ce_encrypt_bit: bad secret key or null output");
  uint32_t acc = 0;
  for (int m = 0; m < kLweN; ++m) {
    out->a[m] = draw_u32(seed, kDomEncA, ctr * kLweN + m);
    acc += out->a[m] * sk.s[m];
  }
  acc += draw_noise(seed, kDomEncNoise, ctr, kSigmaLwe);
  acc += bit ? kMuEighth : 0u - kMuEighth;
  out->b = acc;
  return CE_OK;
}

extern "C" int ce_decrypt_bit(const void *secret, const ce_lwe *c) {
  SecretView sk;
  if (!c || !view_secret(secret, &sk))
    return set_error(CE_EINVAL, "ce_decrypt_bit: bad secret key or null ciphertext");
  uint32_t phase = c->b;
  for (int m = 0; m < kLweN; ++m) phase -= c->a[m] * sk.s[m];
  return static_cast<int32_t>(phase) > 0 ? 1 : 0;
}
