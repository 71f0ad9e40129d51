// Integer-logic peak probe: the denominator of the keystream kernel's
// roofline.  Every thread runs eight independent chains of 3-input LOP3
// (inline PTX so that nothing folds); each block measures its own SM-cycle
// count with clock64.  ops per SM per cycle = ops of the resident blocks on
// one SM / cycles, independent of the clock the GPU ran at.
//
// Bare-clock probe: the keystream kernel's clock loop without any output,
// the ceiling its clock warps can reach.
#include <cuda_runtime.h>

#include <vector>

#include "../../include/grain.h"
#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "grain_clock.cuh"

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

// One group per thread: load 200 words (word-major, G words apart), run
// `clocks` keystream clocks folding every z word into an accumulator, write
// the state and the accumulator back (so nothing is dead code).
__global__ void __launch_bounds__(128, 1)
    clock_probe_kernel(uint32_t *state, uint32_t *acc_out, int clocks, long long *cycles) {
  const uint32_t G = gridDim.x * blockDim.x;
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t r[mickey::kReg], s[mickey::kReg];
#pragma unroll
  for (int i = 0; i < mickey::kReg; ++i) {
    r[i] = state[size_t(i) * G + g];
    s[i] = state[size_t(mickey::kReg + i) * G + g];
  }
  __syncthreads();
  const long long t0 = clock64();
  uint32_t acc = 0;
#pragma unroll 1
  for (int c = 0; c < clocks; c += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc = mickey::lop3<0x96>(acc, r[0], s[0]);
      mickey::clock_kg<false, false>(r, s, 0u, 0u);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
#pragma unroll
  for (int i = 0; i < mickey::kReg; ++i) {
    state[size_t(i) * G + g] = r[i];
    state[size_t(mickey::kReg + i) * G + g] = s[i];
  }
  acc_out[g] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The bare Grain clock: 64 threads per block, one 32-lane group per thread,
// `bodies` x 80 clocks from an arbitrary state; STORE writes each clock's
// keystream word to shared memory (as the keystream kernel's ring does),
// otherwise the words are folded into an accumulator.
template <bool STORE>
__global__ void __launch_bounds__(mickey::grainc::kGrainThreads)
    grain_clock_probe_kernel(uint32_t *state, int bodies, long long *cycles, uint32_t *sink) {
  using namespace mickey::grainc;
  __shared__ uint32_t zb[kG * kGrainThreads];
  const uint32_t G = gridDim.x * blockDim.x;
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t s[kG], b[kG];
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    s[i] = state[size_t(i) * G + g];
    b[i] = state[size_t(kG + i) * G + g];
  }
  __syncthreads();
  const long long t0 = clock64();
  uint32_t acc = 0;
#pragma unroll 1
  for (int k = 0; k < bodies; ++k) {
    if constexpr (STORE) {
      grain_body<false>(s, b, zb + (threadIdx.x >> 5) * (kG * kRingStride) + (threadIdx.x & 31));
    } else {
      mickey::static_for<0, kG>([&](auto rc) {
        constexpr int R = decltype(rc)::value;
        acc ^= grain_clock<R, false>(s, b);
      });
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if constexpr (STORE) acc = zb[threadIdx.x];
#pragma unroll
  for (int i = 0; i < kG; ++i) acc ^= s[i] ^ b[i];
  sink[g] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" MICKEY_API int grain_probe_clock(int blocks_per_sm, int bodies, int store,
                                            double *ops_per_sm_clk, double *sm_mhz) {
  using namespace mickey::grainc;
  if (blocks_per_sm < 1 || blocks_per_sm > 4 || bodies < 1) return MICKEY_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MICKEY_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MICKEY_E_CUDA;
  const int blocks = sms * blocks_per_sm;
  const size_t G = size_t(blocks) * kGrainThreads;
  uint32_t *state = nullptr, *sink = nullptr;
  long long *cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MICKEY_OK;
  if (cudaMalloc(&state, G * 2 * kG * 4) != cudaSuccess || cudaMalloc(&sink, G * 4) != cudaSuccess ||
      cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MICKEY_E_CUDA;
  } else {
    cudaMemset(state, 0x5a, G * 2 * kG * 4);   // any state that is not all zeros or ones
    auto launch = [&](int n) {
      if (store)
        grain_clock_probe_kernel<true><<<blocks, kGrainThreads>>>(state, n, cyc, sink);
      else
        grain_clock_probe_kernel<false><<<blocks, kGrainThreads>>>(state, n, cyc, sink);
    };
    launch(2);   // warm-up
    cudaEventRecord(e0);
    launch(bodies);
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
      const double ops_sm =
          double(kGrainThreads) * blocks_per_sm * double(bodies) * kG * grain_ops_per_clock(0);
      if (ops_per_sm_clk) *ops_per_sm_clk = ops_sm / double(mx);
      if (sm_mhz) *sm_mhz = double(mx) / (ms * 1e3);
    }
  }
  cudaFree(state);
  cudaFree(sink);
  cudaFree(cyc);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

extern "C" MICKEY_API int mickey_probe_clock(int blocks_per_sm, int clocks, double *ops_per_sm_clk,
                                             double *sm_mhz) {
  if (blocks_per_sm < 1 || blocks_per_sm > 2 || clocks < 4 || clocks % 4) return MICKEY_E_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MICKEY_E_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MICKEY_E_CUDA;
  const int blocks = sms * blocks_per_sm;
  const size_t G = size_t(blocks) * 128;
  uint32_t *state = nullptr, *acc = nullptr;
  long long *cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = MICKEY_OK;
  if (cudaMalloc(&state, G * 200 * 4) != cudaSuccess || cudaMalloc(&acc, G * 4) != cudaSuccess ||
      cudaMalloc(&cyc, blocks * sizeof(long long)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = MICKEY_E_CUDA;
  } else {
    // any state will do: a byte pattern that is neither all zeros nor all ones
    cudaMemset(state, 0x5a, G * 200 * 4);
    clock_probe_kernel<<<blocks, 128>>>(state, acc, 64, cyc);  // warm-up
    cudaEventRecord(e0);
    clock_probe_kernel<<<blocks, 128>>>(state, acc, clocks, cyc);
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
      const double ops_sm = 128.0 * blocks_per_sm * double(clocks) * mickey::ops_per_clock(false);
      if (ops_per_sm_clk) *ops_per_sm_clk = ops_sm / double(mx);
      if (sm_mhz) *sm_mhz = double(mx) / (ms * 1e3);
    }
  }
  cudaFree(state);
  cudaFree(acc);
  cudaFree(cyc);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

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
