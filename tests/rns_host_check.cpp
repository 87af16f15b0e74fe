// Host build of the blind rotation's two-prime transform (rns_ntt.cuh) for
// the CPU test suite: runs the 128-thread transform phases one thread after
// another, exactly as the device kernel orders them between barriers, with
// every lazy bound of the arithmetic checked (RNS_RANGE_CHECK).
//
// Input (binary, stdin):  digits int32 [3][2][1024] (level, component, n),
//                         keys uint32 [3][2][2][1024] (level, component, output, n).
// Output (binary, stdout): uint32 [2][1024] = sum over level and component of
//                         digits * keys in Z_{2^32}[X]/(X^1024 + 1), then one
//                         uint32 with the number of violated bounds and one
//                         with the number of forward-transform positions that
//                         differ from a direct evaluation (first key pair).
#include <cstdint>
#include <cstdio>
#include <vector>

static long g_bad = 0;
inline void rns_range_check(bool ok) { g_bad += ok ? 0 : 1; }
#define RNS_RANGE_CHECK
#include "../paper_2101_03403_gb300/csrc/rns_ntt.cuh"

using namespace rns;

static const uint32_t kPr[2] = {P<0>(), P<1>()};

static void tables(std::vector<uint4> &tw) {
  tw.assign(kTwEntries, uint4{});
  const uint32_t roots[2] = {Psi<0>(), Psi<1>()};
  for (int q = 0; q < 2; ++q) {
    const uint32_t p = kPr[q], psi = roots[q], pinv = invm(psi, p), n_inv = invm(1024, p);
    for (int k2 = 0; k2 < 16; ++k2)
      for (int n1 = 0; n1 < 64; ++n1) {
        const uint64_t e = uint64_t(2 * k2 + 1) * n1;
        const uint32_t wf = powm(psi, e, p), wi = mulm(powm(pinv, e, p), n_inv, p);
        uint4 &F = tw[k2 * 64 + n1], &I = tw[1024 + k2 * 64 + n1];
        (q ? F.z : F.x) = wf;
        (q ? F.w : F.y) = shoup_of(wf, p);
        (q ? I.z : I.x) = wi;
        (q ? I.w : I.y) = shoup_of(wi, p);
      }
    for (int a = 0; a < 8; ++a)
      for (int c = 0; c < 8; ++c) {
        const uint32_t wf = powm(psi, 32u * a * c, p), wi = powm(pinv, 32u * a * c, p);
        uint4 &F = tw[kTwC1Fwd + a * 8 + c], &I = tw[kTwC1Inv + a * 8 + c];
        (q ? F.z : F.x) = wf;
        (q ? F.w : F.y) = shoup_of(wf, p);
        (q ? I.z : I.x) = wi;
        (q ? I.w : I.y) = shoup_of(wi, p);
      }
  }
}

// Forward pair transform: in[q][poly][n] (values in [0, 2p)) -> X[t][q][poly][d].
static void forward2(const std::vector<uint4> &tw, const uint32_t (*in)[2][1024],
                     uint32_t (*X)[2][2][8]) {
  std::vector<uint2> buf(kBufWords);
  for (int t = 0; t < 128; ++t) {
    const int Pp = t >> 6, n1 = t & 63;
    uint32_t v[2][16];
    for (int q = 0; q < 2; ++q)
      for (int n2 = 0; n2 < 16; ++n2) v[q][n2] = in[q][Pp][n1 + 64 * n2];
    for (int n2 = 1; n2 < 16; ++n2) {
      v[0][n2] = pretwist<0>(v[0][n2], n2);
      v[1][n2] = pretwist<1>(v[1][n2], n2);
    }
    fwd_phase_a(v, buf.data(), t, tw.data());
  }
  for (int t = 0; t < 128; ++t) fwd_phase_c1(buf.data(), t >> 5, t & 31, tw.data() + kTwC1Fwd);
  for (int t = 0; t < 128; ++t) fwd_phase_c2(X[t], buf.data(), t);
}

int main() {
  static int32_t dig[3][2][1024];
  static uint32_t key[3][2][2][1024];
  if (fread(dig, sizeof dig, 1, stdin) != 1 || fread(key, sizeof key, 1, stdin) != 1) return 2;
  std::vector<uint4> tw;
  tables(tw);

  // Keys to the transform domain: reduced, Montgomery form (as at admission).
  static uint32_t KX[3][2][128][2][2][8];
  long direct_bad = 0;
  for (int l = 0; l < 3; ++l)
    for (int c = 0; c < 2; ++c) {
      static uint32_t kin[2][2][1024];
      for (int q = 0; q < 2; ++q)
        for (int o = 0; o < 2; ++o)
          for (int n = 0; n < 1024; ++n)
            kin[q][o][n] = q ? from_i32<1>(int32_t(key[l][c][o][n]))
                             : from_i32<0>(int32_t(key[l][c][o][n]));
      forward2(tw, kin, KX[l][c]);
      if (l == 0 && c == 0)  // forward transform vs its definition
        for (int t = 0; t < 128; ++t)
          for (int d = 0; d < 8; ++d) {
            const int k = (t & 15) + 16 * ((t >> 4) + 8 * d);
            for (int q = 0; q < 2; ++q)
              for (int o = 0; o < 2; ++o) {
                const uint32_t p = kPr[q], root = q ? Psi<1>() : Psi<0>();
                const uint32_t base = powm(root, 2 * k + 1, p);
                uint64_t s = 0;
                uint32_t w = 1;
                for (int n = 0; n < 1024; ++n) {
                  s = (s + uint64_t(kin[q][o][n]) * w) % p;
                  w = mulm(w, base, p);
                }
                if (KX[l][c][t][q][o][d] % p != s) ++direct_bad;
              }
          }
      for (int t = 0; t < 128; ++t)
        for (int o = 0; o < 2; ++o)
          for (int d = 0; d < 8; ++d) {
            KX[l][c][t][0][o][d] = fold<0, 1>(to_mont<0>(KX[l][c][t][0][o][d]));
            KX[l][c][t][1][o][d] = fold<1, 1>(to_mont<1>(KX[l][c][t][1][o][d]));
          }
    }

  // One CMux step's external product, accumulated as the kernel does: the
  // six key products of an output position summed unreduced in 64 bits,
  // then one Montgomery reduction.
  static uint64_t XL[128][2][2][8];
  static uint32_t X[128][2][2][8];
  for (int l = 0; l < 3; ++l) {
    static uint32_t din[2][2][1024];
    static uint32_t Y[128][2][2][8];
    for (int q = 0; q < 2; ++q)
      for (int c = 0; c < 2; ++c)
        for (int n = 0; n < 1024; ++n) din[q][c][n] = uint32_t(dig[l][c][n] + int32_t(kPr[q]));
    forward2(tw, din, Y);
    for (int t = 0; t < 128; ++t)
      for (int o = 0; o < 2; ++o)
        for (int d = 0; d < 8; ++d) {
          XL[t][0][o][d] += uint64_t(Y[t][0][0][d]) * KX[l][0][t][0][o][d] +
                            uint64_t(Y[t][0][1][d]) * KX[l][1][t][0][o][d];
          XL[t][1][o][d] += uint64_t(Y[t][1][0][d]) * KX[l][0][t][1][o][d] +
                            uint64_t(Y[t][1][1][d]) * KX[l][1][t][1][o][d];
        }
  }
  for (int t = 0; t < 128; ++t)
    for (int o = 0; o < 2; ++o)
      for (int d = 0; d < 8; ++d) {
        X[t][0][o][d] = redc<0>(XL[t][0][o][d]);
        X[t][1][o][d] = redc<1>(XL[t][1][o][d]);
        rns_range_check(X[t][0][o][d] < 7 * kPr[0] && X[t][1][o][d] < 7 * kPr[1]);
      }
  std::vector<uint2> buf(kBufWords);
  for (int t = 0; t < 128; ++t) inv_phase_c2(X[t], buf.data(), t);
  for (int t = 0; t < 128; ++t) inv_phase_c1(buf.data(), t >> 5, t & 31, tw.data() + kTwC1Inv);
  static uint32_t out[2][1024];
  for (int t = 0; t < 128; ++t) {
    const int Pp = t >> 6, n1 = t & 63;
    uint32_t v[2][16];
    inv_phase_a(v, buf.data(), t, tw.data() + kTwInv);
    for (int n2 = 0; n2 < 16; ++n2) out[Pp][n1 + 64 * n2] = lift32(v[0][n2], v[1][n2]);
  }
  fwrite(out, sizeof out, 1, stdout);
  const uint32_t tail[2] = {uint32_t(g_bad), uint32_t(direct_bad)};
  fwrite(tail, sizeof tail, 1, stdout);
  return 0;
}
