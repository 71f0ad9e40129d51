// Integer-logic peak probe: the denominator of the keystream kernel's
// roofline.  Every thread runs eight independent chains of 3-input LOP3
// (inline PTX so that nothing folds); each block measures its own SM-cycle
// count with clock64.  ops per SM per cycle = ops of the resident blocks on
// one SM / cycles, independent of the clock the GPU ran at.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/mickey.h"

namespace {

constexpr int kChains = 8;
constexpr int kInner = 16;

__global__ void lop3_probe_kernel(uint32_t seed, int iters, uint32_t *sink,
                                  long long *cycles) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed * (threadIdx.x + 1) + c;
  const uint32_t b = seed ^ 0x9e3779b9u, d = seed + 0x7f4a7c15u;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kInner; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c)
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[c]) : "r"(b), "r"(d));
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) x ^= a[c];
  if (x == 0x12345678u) sink[blockIdx.x] = x;  // keep the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" MICKEY_API int mickey_probe_lop3(int blocks_per_sm, int threads, int iters,
                                            double *ops_per_sm_clk, double *sm_mhz,
                                            double *tops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MICKEY_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MICKEY_E_CUDA;
  if (blocks_per_sm <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return MICKEY_E_ARG;
  const int blocks = sms * blocks_per_sm;
  uint32_t *sink = nullptr;
  long long *cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MICKEY_OK;
  if (cudaMalloc(&sink, blocks * 4) != cudaSuccess ||
      cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MICKEY_E_CUDA;
  } else {
    lop3_probe_kernel<<<blocks, threads>>>(1u, iters / 10 + 1, sink, cyc);  // warm-up
    cudaEventRecord(e0);
    lop3_probe_kernel<<<blocks, threads>>>(1u, iters, sink, cyc);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = MICKEY_E_CUDA;
    } else {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      std::vector<long long> h(blocks);
      cudaMemcpy(h.data(), cyc, blocks * sizeof(long long), cudaMemcpyDeviceToHost);
      long long mx = 0;
      for (long long c : h) mx = c > mx ? c : mx;
      const double ops_block = double(threads) * iters * kInner * kChains;
      const double per_sm = ops_block * blocks_per_sm;
      if (ops_per_sm_clk) *ops_per_sm_clk = per_sm / double(mx);
      if (sm_mhz) *sm_mhz = double(mx) / (ms * 1e3);
      if (tops) *tops = ops_block * blocks / (ms * 1e-3) / 1e12;
    }
  }
  cudaFree(sink);
  cudaFree(cyc);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}
