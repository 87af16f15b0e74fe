// Integer pipe rate probe (sm_103a): independent dependency chains per
// thread, two 512-thread blocks per SM, per-block clock64 timing.  Reports
// PTX operations per clock per SM for 32-bit multiply-add, 32x32->64
// multiply-add, logic, 64-bit add with carry, plain add, and a multiply-add +
// logic mix (the two integer pipes issue in parallel).
//
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a int_pipe_probe.cu -o probe && ./probe
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

template <int KIND>
__global__ void k(uint32_t *out, long long *cyc, int iters, uint32_t seed) {
  uint32_t a[8], b = seed * 2654435761u + threadIdx.x, c = b ^ 0x9e3779b9u;
  uint64_t w[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = b + j * 77u;
    w[j] = a[j];
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (KIND == 0) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
        if (KIND == 1) asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[j]) : "r"(b), "r"(c + j));
        if (KIND == 2) asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[j]) : "r"(a[(j + 1) & 7]));
        if (KIND == 3)
          asm volatile(
              "{\n\t.reg .u32 lo, hi;\n\tmov.b64 {lo, hi}, %0;\n\tadd.cc.u32 lo, lo, %1;\n\t"
              "addc.u32 hi, hi, %2;\n\tmov.b64 %0, {lo, hi};\n\t}"
              : "+l"(w[j])
              : "r"(b), "r"(c));
        if (KIND == 4) {
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[j]) : "r"(b), "r"(c));
          asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[j]) : "r"(c));
        }
        if (KIND == 5) asm volatile("add.u32 %0, %0, %1;" : "+r"(a[j]) : "r"(b));
      }
    }
  }
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j] + uint32_t(w[j]) + uint32_t(w[j] >> 32);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

int main() {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int threads = 512, iters = 4000, blocks = 2 * sms;
  const char *names[] = {"mad.lo.u32", "mad.wide.u32", "xor.b32", "add.cc + addc (64-bit add)",
                         "mad.lo + xor", "add.u32"};
  const int per_it[] = {1, 1, 1, 2, 2, 1};
  uint32_t *out = nullptr;
  long long *cyc = nullptr;
  cudaMalloc(&out, sizeof(uint32_t) * blocks * threads);
  cudaMalloc(&cyc, sizeof(long long) * blocks);
  long long h[1024];
  if (blocks > 1024) return 1;
  for (int kind = 0; kind < 6; ++kind) {
    for (int rep = 0; rep < 2; ++rep) {
      switch (kind) {
        case 0: k<0><<<blocks, threads>>>(out, cyc, iters, 1); break;
        case 1: k<1><<<blocks, threads>>>(out, cyc, iters, 1); break;
        case 2: k<2><<<blocks, threads>>>(out, cyc, iters, 1); break;
        case 3: k<3><<<blocks, threads>>>(out, cyc, iters, 1); break;
        case 4: k<4><<<blocks, threads>>>(out, cyc, iters, 1); break;
        default: k<5><<<blocks, threads>>>(out, cyc, iters, 1); break;
      }
      cudaDeviceSynchronize();
      cudaMemcpy(h, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
      double mx = 0;
      for (int i = 0; i < blocks; ++i) mx = h[i] > mx ? double(h[i]) : mx;
      const double ops = 2.0 * threads * iters * 32.0 * per_it[kind];  // two blocks per SM
      if (rep) printf("%-28s %.1f PTX ops/clk/SM\n", names[kind], ops / mx);
    }
  }
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
