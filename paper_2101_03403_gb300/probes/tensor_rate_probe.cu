// Tensor-core rate probe for the exact external-product question on sm_103a:
// back-to-back independent mma.sync (int8 m16n8k32 and fp16 m16n8k16) on
// register operands, all SMs, CUDA-event timed.  (tcgen05.mma kind::i8 is
// not available on sm_103a: ptxas rejects it for that target.)
//
//   nvcc -O3 -gencode arch=compute_103a,code=sm_103a tensor_rate_probe.cu -o probe && ./probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
template <int KIND>
__global__ void k(int* out, int iters, uint32_t seed) {
  uint32_t a0 = seed ^ threadIdx.x, a1 = a0 * 3, a2 = a0 * 5, a3 = a0 * 7, b0 = a0 * 11, b1 = a0 * 13;
  int d[4][4] = {};
  float f[4][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (KIND == 0)
        asm volatile("mma.sync.aligned.m16n8k32.row.col.s32.u8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                     : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3]) : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      else
        asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                     : "+f"(f[j][0]), "+f"(f[j][1]), "+f"(f[j][2]), "+f"(f[j][3]) : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
    }
  }
  int s = 0;
  for (int j = 0; j < 4; ++j) for (int q = 0; q < 4; ++q) s += d[j][q] + (int)f[j][q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
int main() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  const int blocks = sms * 4, threads = 256, iters = 20000;
  int* out; cudaMalloc(&out, sizeof(int) * blocks * threads);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int kind = 0; kind < 2; ++kind) {
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0);
      if (kind == 0) k<0><<<blocks, threads>>>(out, iters, 1); else k<1><<<blocks, threads>>>(out, iters, 1);
      cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1);
      const double warps = double(blocks) * threads / 32;
      const double ops = warps * iters * 4 * (kind == 0 ? 16.0 * 8 * 32 * 2 : 16.0 * 8 * 16 * 2);
      if (rep) printf("%s mma.sync: %.3f ms, %.1f TOPS\n", kind == 0 ? "int8 m16n8k32" : "fp16 m16n8k16", ms, ops / ms / 1e9);
    }
  }
  printf("err: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
