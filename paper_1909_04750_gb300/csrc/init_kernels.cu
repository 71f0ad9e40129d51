// Key/IV loading for bitsliced MICKEY 2.0 (Sec. IV-A representation change,
// Sec. IV-D input handler, and the cipher's initialisation).
//
// load_kernel      one thread per 32-lane group: reads the group's 32 keys,
//                  IVs and IV lengths and turns them into bitsliced words
//                  with 32x32 bit-matrix transposes (row-major -> column-
//                  major, Sec. IV-A).  IVs are right-aligned per lane so that
//                  all lanes of a group end their IV phase on the same clock;
//                  a lane with a shorter IV is held still (masked) until its
//                  first IV bit.
// preclock_kernel  one thread per group: zero state, IV clocks, 80 key
//                  clocks, 100 mixing preclocks, all in mixing mode; writes
//                  the 200-word state.
#include "bitslice.cuh"
#include "internal.h"

namespace mickey {
namespace {

__device__ __forceinline__ uint32_t load_be32(const uint8_t *p) {
  return (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16) |
         (uint32_t(p[2]) << 8) | uint32_t(p[3]);
}

// Word k (k = 0 most significant) of the mask selecting the first m bits
// of a 96-bit big-endian bit string.
__device__ __forceinline__ uint32_t prefix_mask(int m, int k) {
  const int lo = 32 * k;
  if (m >= lo + 32) return ~0u;
  if (m <= lo) return 0u;
  return ~0u << (32 - (m - lo));
}

__device__ __forceinline__ uint32_t pick3(uint32_t w0, uint32_t w1,
                                          uint32_t w2, int idx) {
  return idx == 0 ? w0 : idx == 1 ? w1 : idx == 2 ? w2 : 0u;
}

// Word k of the 96-bit big-endian string (w0, w1, w2) moved s bits towards
// higher bit indices (bit b -> bit b + s); 0 <= s <= 80.
__device__ __forceinline__ uint32_t shift96_word(uint32_t w0, uint32_t w1,
                                                 uint32_t w2, int s, int k) {
  const int ws = s >> 5, bs = s & 31;
  const int i_lo = k - ws, i_hi = k - ws - 1;
  const uint32_t lo = i_lo >= 0 ? pick3(w0, w1, w2, i_lo) : 0u;
  const uint32_t hi = i_hi >= 0 ? pick3(w0, w1, w2, i_hi) : 0u;
  return __funnelshift_r(lo, hi, bs);
}

// Instance held by lane slot `slot` (32g + l).
__device__ __forceinline__ uint64_t inst(const LoadArgs &a, uint64_t slot) {
  return a.perm ? uint64_t(a.perm[slot]) : slot;
}

__global__ void __launch_bounds__(kInitThreads) load_kernel(LoadArgs a) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  const uint64_t base = 32ull * g;
  const uint64_t left = a.n - base;
  const int nv = left >= 32 ? 32 : int(left);

  int len[32];
  int max_len = 0, min_len = 80;
#pragma unroll
  for (int l = 0; l < 32; ++l) {
    int v = 0;
    if (l < nv) {
      v = a.iv_lens ? int(min(a.iv_lens[inst(a, base + l)], 1000u)) : 80;
      if (v > 80) {
        atomicOr(a.err, kErrIvLen);
        v = 80;
      }
      max_len = max(max_len, v);
      min_len = min(min_len, v);
    }
    len[l] = v;
  }
  // The IV phase runs a multiple of 4 clocks (the preclock loop handles four
  // clocks per iteration); lanes are right-aligned to that length.
  const int phase = (max_len + 3) & ~3;
#pragma unroll
  for (int l = 0; l < 32; ++l)
    if (l >= nv) len[l] = phase;  // padding lanes: zero inputs, no masking
  const bool mixed = min_len != phase;

  // Key bits: three 32-bit chunks per lane (the third holds bits 64..79).
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;  // row r = lane 31-r, so result bit l = lane l
      uint32_t w = 0;
      if (l < nv) {
        const uint8_t *p = a.keys + inst(a, base + l) * 10 + 4 * q;
        w = q < 2 ? load_be32(p) : (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16);
      }
      m[r] = w;
    }
    transpose32(m);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int row = 32 * q + j;
      if (row < 80) a.scratch[size_t(kKeyRow + row) * a.Gpad + g] = m[j];
    }
  }

  // IV bits, right-aligned: lane l's bit b is consumed at IV clock
  // b + (phase - len[l]); before that the lane is inactive (zero state).
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    if (32 * q >= phase) break;
    uint32_t m[32], act[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;
      const int L = len[l];
      const int sft = phase - L;
      uint32_t w = 0;
      if (l < nv && L > 0) {
        const uint8_t *p = a.ivs + inst(a, base + l) * 10;
        const uint32_t w0 = load_be32(p) & prefix_mask(L, 0);
        const uint32_t w1 = load_be32(p + 4) & prefix_mask(L, 1);
        const uint32_t w2 =
            ((uint32_t(p[8]) << 24) | (uint32_t(p[9]) << 16)) & prefix_mask(L, 2);
        w = shift96_word(w0, w1, w2, sft, q);
      }
      m[r] = w;
      act[r] = prefix_mask(phase, q) & ~prefix_mask(sft, q);
    }
    transpose32(m);
    if (mixed) transpose32(act);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = 32 * q + j;
      if (c < phase) {
        a.scratch[size_t(kIvRow + c) * a.Gpad + g] = m[j];
        if (mixed) a.scratch[size_t(kActRow + c) * a.Gpad + g] = act[j];
      }
    }
  }
  a.scratch[size_t(kScratchRows) * a.Gpad + g] =
      uint32_t(phase) | (mixed ? 0x100u : 0u);
}

constexpr int kPre = 2;  // clocks per loop iteration (IV phase is a multiple of 4)

// kPre clocks per loop iteration: with a single clock per iteration the
// shift of both registers makes every loop-carried word change register,
// which costs copies and spills.
__global__ void __launch_bounds__(kInitThreads) preclock_kernel(PreclockArgs a) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  uint32_t r[kReg], s[kReg];
#pragma unroll
  for (int i = 0; i < kReg; ++i) r[i] = s[i] = 0u;

  const uint32_t info = a.scratch[size_t(kScratchRows) * a.Gpad + g];
  const int phase = int(info & 0xFFu);  // IV clocks, a multiple of 4
  const bool mixed = (info >> 8) & 1u;
  const uint32_t *col = a.scratch + g;
  const size_t P = a.Gpad;

  if (mixed) {
#pragma unroll 1
    for (int c = 0; c < phase; c += kPre) {
#pragma unroll
      for (int u = 0; u < kPre; ++u)
        clock_kg<true, true>(r, s, col[(kIvRow + c + u) * P], col[(kActRow + c + u) * P]);
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < phase; c += kPre) {
#pragma unroll
      for (int u = 0; u < kPre; ++u) clock_kg<true, false>(r, s, col[(kIvRow + c + u) * P], 0u);
    }
  }
#pragma unroll 1
  for (int j = 0; j < 80; j += kPre) {
#pragma unroll
    for (int u = 0; u < kPre; ++u) clock_kg<true, false>(r, s, col[(kKeyRow + j + u) * P], 0u);
  }
#pragma unroll 1
  for (int c = 0; c < 100; c += kPre) {
#pragma unroll
    for (int u = 0; u < kPre; ++u) clock_kg<true, false>(r, s, 0u, 0u);
  }

  uint32_t *st = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    st[size_t(i) * P] = r[i];
    st[size_t(kReg + i) * P] = s[i];
  }
}

}  // namespace

cudaError_t launch_load(const LoadArgs &a, cudaStream_t st) {
  const uint32_t blocks = (a.G + kInitThreads - 1) / kInitThreads;
  load_kernel<<<blocks, kInitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_preclock(const PreclockArgs &a, cudaStream_t st) {
  const uint32_t blocks = (a.G + kInitThreads - 1) / kInitThreads;
  preclock_kernel<<<blocks, kInitThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace mickey
