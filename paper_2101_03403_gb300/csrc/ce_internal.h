// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/cryptoemu.h"

namespace ce {

// Parameter set of the gate-bootstrapping workload (fixed at compile time).
constexpr int kLweN = 500;            // LWE dimension n
constexpr int kLweWords = 501;        // a[500], b
constexpr int kRingN = 1024;          // TRLWE degree N (k = 1)
constexpr int kGadgetL = 3;           // gadget length l
constexpr int kBgBit = 10;            // log2 Bg
constexpr int kKsT = 8;               // key-switch digits t
constexpr int kKsBaseBit = 2;         // log2 key-switch base
constexpr int kKsBase = 4;
constexpr double kSigmaLwe = 1.0 / 32768.0;   // 2^-15
constexpr double kSigmaBsk = 9e-9;
constexpr uint32_t kMuEighth = 0x20000000u;   // +1/8

// Device layouts.
constexpr int kAbarStride = 512;      // uint16 words per gate: abar[500], bbar, pad
constexpr int kKskRow = 512;          // padded KSK row: a[500], b, 11 zero words
constexpr int kSlotWords = 512;       // engine arena slot: a[500], b, padding
// Key-switching key on the device keeps only v = 1..3 (v = 0 adds nothing):
// [j][q][v-1][kKskRow] uint32.
constexpr uint64_t kKskDevWords = uint64_t(kRingN) * kKsT * 3 * kKskRow;
// Bootstrapping key in the transform domain: [i][p][4][4][128][2] uint64
// with 4 = (TRGSW half c, output component o) and [4][128][2] = (register
// pair d/2, thread, d%2).
constexpr int kChunkWords = 4 * 8 * 128;                  // 4096 uint64 = 32 KB
constexpr uint64_t kBskNttWords = uint64_t(kLweN) * kGadgetL * kChunkWords;

ce_status set_error(ce_status code, const std::string &msg);

// Device allocations of the library, counted (ce_device_alloc_count).
cudaError_t dev_malloc(void **p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T **p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
void dev_free(void *p);

}  // namespace ce
