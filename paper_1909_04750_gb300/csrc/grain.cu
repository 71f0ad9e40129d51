// Bitsliced Grain (version 1) keystream generation: the paper's second
// stream cipher (Sec. II-C-3: an 80-bit LFSR and an 80-bit NFSR shifted
// together each clock, 80-bit key, 64-bit IV, 160 initialisation clocks),
// in the column-major representation of Sec. IV-A: a 32-bit word holds the
// same register bit of 32 instances, one thread clocks a 32-lane group.
//
// State: s[0..79] (LFSR) and b[0..79] (NFSR), 160 words in registers.  The
// shift of both registers is never executed: slot (R + i) % 80 holds s_{i}
// when R clocks have passed (mod 80), and a clock overwrites slot R (the
// oldest bit) with the new bit s_{i+80}; unrolling 80 clocks brings the
// mapping back to the start (register renaming, Sec. IV-C).
//
// Per clock, with 3-input logic instructions (lop3.b32):
//   LFSR   s_{i+80} = s62+s51+s38+s23+s13+s0                        3 ops
//   NFSR   b_{i+80} = s0 + g(b): 12 linear terms and 11 products of 2 to 6
//          taps, with the partial products b63b60, b37b33, b15b9, b60b52,
//          b52b45, b33b28b21 and b63b45b28 shared                   23 ops
//   output z = b1+b2+b4+b10+b31+b43+b56 + h(s3,s25,s46,s64,b63), h written
//          as A + x2*B with A = x1+x4+x3(x0+x4), B = x3+x4(x1+x3)+x0(x1+x3+x4)
//                                                                   11 ops
//   init   z is added into both new bits (into the LFSR's last XOR)  +1
// Keystream words go to a ring of 160 words per thread in shared memory
// (two bodies of 80 clocks fill five 32-clock tiles); after each body the
// finished tiles are emitted: as they are (bitsliced layout) or, for
// row-major bytes, transposed by the two-pass in-place block swaps also used
// for MICKEY and bit-reversed, since Grain's bytes hold the first keystream
// bit in the least significant bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/grain.h"
#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "internal.h"

namespace mickey {
namespace {

constexpr int kG = 80;               // register length
constexpr int kGrainThreads = 64;    // groups per block
constexpr int kRing = 160;           // keystream words per thread in the ring

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x96>(a, b, c);
}
__device__ __forceinline__ uint32_t and3(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x80>(a, b, c);
}
__device__ __forceinline__ uint32_t xand(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x78>(a, b, c);   // a ^ (b & c)
}

// One clock at rotation R (compile-time): returns z of the current state
// and replaces slot R of both registers by the new bits.  The XOR sums are
// balanced trees (at most five dependent steps to the new NFSR bit, four to
// z), so that the instructions of one clock can issue back to back.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t grain_clock(uint32_t (&s)[kG], uint32_t (&b)[kG]) {
#define S(i) s[(R + (i)) % kG]
#define B(i) b[(R + (i)) % kG]
  // output: z = b1+b2+b4+b10+b31+b43+b56 + h(x0..x4),
  // h = A + x2 B, A = x1+x4+x3(x0+x4), B = x3+x4(x1+x3)+x0(x1+x3+x4)
  const uint32_t x0 = S(3), x1 = S(25), x2 = S(46), x3 = S(64), x4 = B(63);
  const uint32_t t1 = xor3(B(1), B(2), B(4));
  const uint32_t t2 = xor3(B(10), B(31), B(43));
  const uint32_t u0 = xor3(x1, x4, B(56));
  const uint32_t t = x0 ^ x4;
  const uint32_t w = x1 ^ x3;
  const uint32_t v = xor3(x1, x3, x4);
  const uint32_t u = xor3(t1, t2, u0);                 // x1 + x4 + (b sum)
  const uint32_t c = xand(x3, x4, w);                  // x3 + x4(x1 + x3)
  const uint32_t a = xand(u, x3, t);                   // A + (b sum)
  const uint32_t bb = xand(c, x0, v);                  // B
  const uint32_t z = xand(a, x2, bb);                  // A + x2 B + (b sum)
  // LFSR: s62+s51+s38+s23+s13+s0 (+ z while initialising)
  const uint32_t la = xor3(S(62), S(51), S(38));
  const uint32_t lb = xor3(S(23), S(13), S(0));
  const uint32_t ns = INIT ? xor3(la, lb, z) : la ^ lb;
  // NFSR: s0 + g(b), the 23 terms in a tree
  const uint32_t p1 = B(63) & B(60);
  const uint32_t p2 = B(37) & B(33);
  const uint32_t p3 = B(15) & B(9);
  const uint32_t q = B(60) & B(52);
  const uint32_t r = B(52) & B(45);
  const uint32_t p5 = and3(B(33), B(28), B(21));
  const uint32_t p6 = and3(B(63), B(45), B(28));
  const uint32_t l1 = xor3(B(62), B(60), B(52));
  const uint32_t l2 = xor3(B(45), B(37), B(33));
  const uint32_t l3 = xor3(B(28), B(21), B(14));
  const uint32_t l4 = xor3(B(9), B(0), S(0));
  const uint32_t m1 = xor3(l1, l2, l3);                 // the linear terms ...
  const uint32_t m2 = xor3(l4, p1, p2);                 // ... s0, b63b60, b37b33
  const uint32_t m3 = xand(p3, q, B(45));               // b15b9, b60b52b45
  const uint32_t m4 = xand(p5, p6, B(9));               // b33b28b21, b63b45b28b9
  const uint32_t t8 = and3(p1, B(21), B(15));           // b63b60b21b15
  const uint32_t t9 = and3(p1, r, B(37));               // b63b60b52b45b37
  const uint32_t t11 = and3(r, B(37), p5);              // b52b45b37b33b28b21
  const uint32_t n1 = xor3(m1, m2, m3);
  const uint32_t n2 = xand(m4, q, p2);                  // b60b52b37b33
  const uint32_t n3 = xor3(t8, t9, t11);
  const uint32_t n4 = xand(n2, p5, p3);                 // b33b28b21b15b9
  uint32_t nb = xor3(n1, n4, n3);
  if (INIT) nb ^= z;
  S(0) = ns;   // slot R: the oldest bit becomes the newest
  B(0) = nb;
#undef S
#undef B
  return z;
}

// 80 clocks (one full rotation); keystream word of clock c to zb[c * kGrainThreads].
template <bool INIT>
__device__ __forceinline__ void grain_body(uint32_t (&s)[kG], uint32_t (&b)[kG], uint32_t *zb) {
  static_for<0, kG>([&](auto rc) {
    constexpr int R = decltype(rc)::value;
    const uint32_t z = grain_clock<R, INIT>(s, b);
    if constexpr (!INIT) zb[R * kGrainThreads] = z;
  });
}

// One clock with the registers physically shifted (rotation stays 0): the
// tail of a call, fewer than 80 clocks.
__device__ __forceinline__ uint32_t grain_clock_shift(uint32_t (&s)[kG], uint32_t (&b)[kG]) {
  const uint32_t s0 = s[0], b0 = b[0];
  const uint32_t z = grain_clock<0, false>(s, b);   // writes the new bits to slot 0
  const uint32_t ns = s[0], nb = b[0];
  s[0] = s0;
  b[0] = b0;
  static_for<0, kG - 1>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    s[i] = s[i + 1];
    b[i] = b[i + 1];
  });
  s[kG - 1] = ns;
  b[kG - 1] = nb;
  return z;
}

struct GrainArgs {
  uint32_t *state;      // 160 x Gpad words: s0..s79 then b0..b79
  uint32_t G, Gpad;
  uint64_t n;
  uint64_t n_bits;
  void *out;
  uint32_t last_mask;   // valid lanes of the last group
};

// Row staging of the bytes layout: the transposed words of 8 consecutive
// tiles per lane, [lane][thread][8] words, so that each row goes out as one
// whole 32-byte sector (two 16-byte stores) instead of 4-byte pieces.
constexpr int kStage = 8;

// Emit the 32-clock tile k of the call (clocks 32k .. 32k+nb-1) held in zb
// (word c = clock 32k + c, bit l = lane l) of group g.  Bitsliced: stored as
// it is.  Bytes: transposed and staged in rb; the staged tiles are written
// out after the last tile of each aligned block of 8 and after the call's
// last tile.
template <int LAYOUT>
__device__ __forceinline__ void grain_emit(uint32_t *zb, uint32_t *rb, const GrainArgs &a,
                                           uint32_t g, uint64_t k, int nb, uint32_t mask) {
  constexpr int T = kGrainThreads;
  const uint64_t t0 = k << 5;
  if constexpr (LAYOUT == MICKEY_LAYOUT_BITSLICED_U32) {
    uint32_t *o = static_cast<uint32_t *>(a.out) + size_t(g) * a.n_bits + t0;
    if (nb == 32 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint4 v;
        v.x = zb[(4 * j + 0) * T] & mask;
        v.y = zb[(4 * j + 1) * T] & mask;
        v.z = zb[(4 * j + 2) * T] & mask;
        v.w = zb[(4 * j + 3) * T] & mask;
        reinterpret_cast<uint4 *>(o)[j] = v;
      }
    } else {
      for (int c = 0; c < nb; ++c) o[c] = zb[c * T] & mask;
    }
  } else {
    // pass 1: block swaps of size 4, 2, 1 within each 8 rows
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = zb[(8 * j + q) * T];
      swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
      swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
      swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
      swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
      swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
      swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
      for (int q = 0; q < 8; ++q) zb[(8 * j + q) * T] = v[q];
    }
    // pass 2: block swaps of size 16 and 8; row k + 8q is lane 31 - k - 8q,
    // its word has the tile's first clock in bit 31, which Grain's bytes
    // take in bit 0 (bit reversal)
    const int slot = int(k & (kStage - 1));
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = zb[(r + 8 * q) * T];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes<false>(v[0], v[1]);
      swap_bytes<false>(v[2], v[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) rb[(31 - r - 8 * q) * (T * kStage) + slot] = __brev(v[q]);
    }
    const bool last = t0 + uint64_t(nb) >= a.n_bits;
    if (slot == kStage - 1 || last) {
      // write tiles k - slot .. k of every valid lane
      const uint32_t pitch = uint32_t((a.n_bits + 7) >> 3);
      const uint64_t kA = k - uint64_t(slot);
      uint8_t *base = static_cast<uint8_t *>(a.out) + 32ull * g * pitch + kA * 4;
      const bool sector = slot == kStage - 1 && nb == 32 && (pitch & 15u) == 0 &&
                          (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
#pragma unroll 1
      for (int l = 0; l < 32; ++l) {
        if (!((mask >> l) & 1u)) continue;
        const uint32_t *src = rb + l * (T * kStage);
        uint8_t *o = base + uint64_t(uint32_t(l) * pitch);
        if (sector) {
          reinterpret_cast<uint4 *>(o)[0] = reinterpret_cast<const uint4 *>(src)[0];
          reinterpret_cast<uint4 *>(o)[1] = reinterpret_cast<const uint4 *>(src)[1];
        } else {
          const uint64_t bytes = ((kA << 5) + ((uint64_t(slot) << 5) + uint64_t(nb)) + 7) / 8 -
                                 ((kA << 5) >> 3);
          for (uint64_t by = 0; by < bytes; ++by) o[by] = uint8_t(src[by >> 2] >> (8 * (by & 3)));
        }
      }
    }
  }
}

template <int LAYOUT>
__global__ void __launch_bounds__(kGrainThreads) grain_keystream_kernel(GrainArgs a) {
  // shared memory: the keystream ring (kRing words per thread, [word][thread])
  // and, for the bytes layout, the row staging ([lane][thread][8])
  extern __shared__ __align__(16) uint32_t ring[];
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  const size_t P = a.Gpad;
  uint32_t s[kG], b[kG];
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    s[i] = a.state[size_t(i) * P + g];
    b[i] = a.state[size_t(kG + i) * P + g];
  }
  const uint32_t mask = g == a.G - 1 ? a.last_mask : ~0u;
  uint32_t *zb = ring + threadIdx.x;
  uint32_t *rb = ring + kRing * kGrainThreads + threadIdx.x * kStage;
  const uint64_t full = a.n_bits / kG;       // whole bodies of 80 clocks
  uint64_t emitted = 0;                      // tiles emitted so far
#pragma unroll 1
  for (uint64_t j = 0; j < full; ++j) {
    grain_body<false>(s, b, zb + (j & 1) * kG * kGrainThreads);
    const uint64_t done = (j + 1) * kG;
#pragma unroll 1
    for (; (emitted + 1) * 32 <= done; ++emitted)
      grain_emit<LAYOUT>(zb + ((emitted * 32) % kRing) * kGrainThreads, rb, a, g, emitted, 32,
                         mask);
  }
  const int rem = int(a.n_bits - full * kG);
  if (rem) {
    uint32_t *zt = zb + (full & 1) * kG * kGrainThreads;
#pragma unroll 1
    for (int c = 0; c < rem; ++c) zt[c * kGrainThreads] = grain_clock_shift(s, b);
  }
#pragma unroll 1
  for (; emitted * 32 < a.n_bits; ++emitted) {
    const int nb = int(min(uint64_t(32), a.n_bits - emitted * 32));
    uint32_t *zt = zb + ((emitted * 32) % kRing) * kGrainThreads;
    for (int c = nb; c < 32; ++c) zt[c * kGrainThreads] = 0u;   // past the call's last clock
    grain_emit<LAYOUT>(zt, rb, a, g, emitted, nb, mask);
  }
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    a.state[size_t(i) * P + g] = s[i];
    a.state[size_t(kG + i) * P + g] = b[i];
  }
}

// ---------------------------------------------------------------- init

struct GrainInitArgs {
  const uint8_t *keys;  // n x 10
  const uint8_t *ivs;   // n x 8
  uint64_t n;
  uint32_t G, Gpad;
  uint32_t *state;
};

constexpr int kInitT = 64;                   // groups per block
constexpr int kKeyWords = 81;                // 80 words of 32 keys + a spare (odd stride)
constexpr int kIvWords = 65;                 // 64 words of 32 IVs + a spare

// Copy `bytes` bytes of src into rows of row_bytes bytes, stride_words apart.
__device__ __forceinline__ void stage(const uint8_t *src, uint64_t bytes, uint32_t *dst,
                                      int row_bytes, int stride_words) {
  const int row_words = row_bytes / 4;
  for (uint64_t w = threadIdx.x; w * 4 < bytes; w += kInitT) {
    uint32_t v;
    if ((reinterpret_cast<uintptr_t>(src) & 3u) == 0 && w * 4 + 4 <= bytes) {
      v = reinterpret_cast<const uint32_t *>(src)[w];
    } else {
      v = 0;
      for (int k = 0; k < 4 && w * 4 + k < bytes; ++k) v |= uint32_t(src[w * 4 + k]) << (8 * k);
    }
    dst[(w / row_words) * stride_words + w % row_words] = v;
  }
}

// Little-endian 32 bits at byte offset o of a staged row, bit-reversed: bit
// (31 - j) of the result is bit j of the byte string from o on (least
// significant bit of each byte first), i.e. the row of a 32x32 transpose.
__device__ __forceinline__ uint32_t lsb_chunk(const uint32_t *row, int o) {
  const uint32_t w0 = row[o >> 2], w1 = row[(o >> 2) + 1];
  return __brev(__funnelshift_r(w0, w1, 8 * (o & 3)));
}

__global__ void __launch_bounds__(kInitT) grain_init_kernel(GrainInitArgs a) {
  __shared__ uint32_t ks[kInitT * kKeyWords], vs[kInitT * kIvWords];
  const uint64_t first = 32ull * blockIdx.x * kInitT;
  const uint64_t count = min(uint64_t(32) * kInitT, a.n - first);
  stage(a.keys + first * 10, count * 10, ks, 320, kKeyWords);
  stage(a.ivs + first * 8, count * 8, vs, 256, kIvWords);
  __syncthreads();
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  const uint64_t left = a.n - 32ull * g;
  const int nv = left >= 32 ? 32 : int(left);
  const uint32_t *krow = ks + threadIdx.x * kKeyWords, *vrow = vs + threadIdx.x * kIvWords;
  uint32_t s[kG], b[kG];
  // key bits 32q .. 32q+31 of the 32 lanes: row r of the matrix is lane
  // 31 - r, so that after the transpose word j has bit l = that bit of lane l
  static_for<0, 3>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    uint32_t m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;
      uint32_t v = l < nv ? lsb_chunk(krow, 10 * l + 4 * q) : 0u;
      if (q == 2) v &= 0xFFFF0000u;           // bits 64..79 only
      m[r] = v;
    }
    transpose32(m);
    static_for<0, 32>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      if constexpr (32 * q + j < kG) b[32 * q + j] = m[j];
    });
  });
  static_for<0, 2>([&](auto qc) {
    constexpr int q = decltype(qc)::value;
    uint32_t m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;
      m[r] = l < nv ? lsb_chunk(vrow, 8 * l + 4 * q) : 0u;
    }
    transpose32(m);
    static_for<0, 32>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      s[32 * q + j] = m[j];
    });
  });
#pragma unroll
  for (int i = 64; i < kG; ++i) s[i] = ~0u;    // s64..s79 = 1
  grain_body<true>(s, b, nullptr);             // 160 clocks, z fed back
  grain_body<true>(s, b, nullptr);
  const size_t P = a.Gpad;
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    a.state[size_t(i) * P + g] = s[i];
    a.state[size_t(kG + i) * P + g] = b[i];
  }
}

template <int LAYOUT>
cudaError_t launch_grain_layout(const GrainArgs &a, cudaStream_t st) {
  const size_t smem = size_t(kRing) * kGrainThreads * 4 +
                      (LAYOUT == MICKEY_LAYOUT_BYTES ? size_t(32) * kGrainThreads * kStage * 4 : 0);
  cudaError_t e = cudaFuncSetAttribute(grain_keystream_kernel<LAYOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  grain_keystream_kernel<LAYOUT><<<(a.G + kGrainThreads - 1) / kGrainThreads, kGrainThreads, smem,
                                   st>>>(a);
  return cudaGetLastError();
}

// Logic ops per clock per 32-lane group, as written above (keystream clock
// including z, or an initialisation clock).
constexpr int kGrainOps = 11 + 3 + 23;
constexpr int kGrainInitOps = kGrainOps + 1;

}  // namespace
}  // namespace mickey

using namespace mickey;

struct grain_streams {
  size_t n = 0;
  uint32_t G = 0, Gpad = 0;
  uint32_t *d_state = nullptr;
  uint8_t *d_inputs = nullptr;   // host inputs staged: keys (10n), ivs (8n)
  cudaStream_t stream = nullptr;
  uint64_t pos = 0;
};

namespace {

int grain_fail(int code, const char *msg) { return set_error(code, msg); }

void grain_release(grain_streams *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->d_state);
  cudaFree(s->d_inputs);
  delete s;
}

size_t grain_out_bytes(size_t n, uint64_t n_bits, int layout) {
  if (layout == MICKEY_LAYOUT_BITSLICED_U32) return size_t((n + 31) / 32 * n_bits * 4);
  if (layout == MICKEY_LAYOUT_BYTES) return size_t(n * ((n_bits + 7) / 8));
  return 0;
}

}  // namespace

extern "C" {

MICKEY_API grain_streams *grain_init_streams(const void *keys, const void *ivs, size_t n, int mem,
                                             void *cuda_stream) {
  if (!keys || !ivs || n == 0 || n > (size_t(1) << 36) ||
      (mem != MICKEY_MEM_HOST && mem != MICKEY_MEM_DEVICE)) {
    grain_fail(MICKEY_E_ARG, "keys/ivs must not be NULL, 0 < n <= 2^36, mem host or device");
    return nullptr;
  }
  grain_streams *s = new (std::nothrow) grain_streams;
  if (!s) {
    grain_fail(MICKEY_E_OOM, "host allocation failed");
    return nullptr;
  }
  s->n = n;
  s->G = uint32_t((n + 31) / 32);
  s->Gpad = (s->G + 31u) & ~31u;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  const uint8_t *dk = static_cast<const uint8_t *>(keys), *dv = static_cast<const uint8_t *>(ivs);
  bool ok = cudaMalloc(&s->d_state, size_t(2 * kG) * s->Gpad * 4) == cudaSuccess;
  if (ok && mem == MICKEY_MEM_HOST) {
    ok = cudaMalloc(&s->d_inputs, n * 18) == cudaSuccess &&
         cudaMemcpyAsync(s->d_inputs, keys, n * 10, cudaMemcpyHostToDevice, s->stream) ==
             cudaSuccess &&
         cudaMemcpyAsync(s->d_inputs + n * 10, ivs, n * 8, cudaMemcpyHostToDevice, s->stream) ==
             cudaSuccess;
    dk = s->d_inputs;
    dv = s->d_inputs + n * 10;
  }
  if (ok) {
    GrainInitArgs ia{dk, dv, n, s->G, s->Gpad, s->d_state};
    grain_init_kernel<<<(s->G + kInitT - 1) / kInitT, kInitT, 0, s->stream>>>(ia);
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (!ok) {
    grain_release(s);
    grain_fail(MICKEY_E_CUDA, "device allocation, copy or launch failed");
    return nullptr;
  }
  set_error(MICKEY_OK, "");
  return s;
}

MICKEY_API int grain_reset_streams(grain_streams *s, const void *keys, const void *ivs, int mem) {
  if (!s || !keys || !ivs || (mem != MICKEY_MEM_HOST && mem != MICKEY_MEM_DEVICE))
    return grain_fail(MICKEY_E_ARG, "NULL argument or bad memory kind");
  const size_t n = s->n;
  const uint8_t *dk = static_cast<const uint8_t *>(keys), *dv = static_cast<const uint8_t *>(ivs);
  if (mem == MICKEY_MEM_HOST) {
    if (!s->d_inputs && cudaMalloc(&s->d_inputs, n * 18) != cudaSuccess)
      return grain_fail(MICKEY_E_OOM, "input staging");
    if (cudaMemcpyAsync(s->d_inputs, keys, n * 10, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(s->d_inputs + n * 10, ivs, n * 8, cudaMemcpyHostToDevice, s->stream) !=
            cudaSuccess)
      return grain_fail(MICKEY_E_CUDA, "key/IV upload");
    dk = s->d_inputs;
    dv = s->d_inputs + n * 10;
  }
  GrainInitArgs ia{dk, dv, n, s->G, s->Gpad, s->d_state};
  grain_init_kernel<<<(s->G + kInitT - 1) / kInitT, kInitT, 0, s->stream>>>(ia);
  if (cudaGetLastError() != cudaSuccess) return grain_fail(MICKEY_E_CUDA, "grain init launch");
  s->pos = 0;
  return set_error(MICKEY_OK, "");
}

MICKEY_API int grain_generate(grain_streams *s, uint64_t n_bits, void *out, int layout) {
  if (!s || !out || n_bits == 0) return grain_fail(MICKEY_E_ARG, "NULL argument or n_bits == 0");
  if (n_bits > kMaxBitsPerCall) return grain_fail(MICKEY_E_ARG, "n_bits per call is limited to 2^34");
  if (layout != MICKEY_LAYOUT_BITSLICED_U32 && layout != MICKEY_LAYOUT_BYTES)
    return grain_fail(MICKEY_E_LAYOUT, "Grain takes the bitsliced or the bytes layout");
  if (layout == MICKEY_LAYOUT_BITSLICED_U32 && (reinterpret_cast<uintptr_t>(out) & 3u))
    return grain_fail(MICKEY_E_ARG, "bitsliced output must be 4-byte aligned");
  const uint32_t tail = uint32_t(s->n & 31u);
  GrainArgs a{s->d_state, s->G, s->Gpad, s->n, n_bits, out, tail ? (1u << tail) - 1u : ~0u};
  const cudaError_t e = layout == MICKEY_LAYOUT_BYTES
                            ? launch_grain_layout<MICKEY_LAYOUT_BYTES>(a, s->stream)
                            : launch_grain_layout<MICKEY_LAYOUT_BITSLICED_U32>(a, s->stream);
  if (e != cudaSuccess) return grain_fail(MICKEY_E_CUDA, "grain keystream launch");
  s->pos += n_bits;
  return set_error(MICKEY_OK, "");
}

MICKEY_API size_t grain_output_bytes(size_t n, uint64_t n_bits, int layout) {
  return grain_out_bytes(n, n_bits, layout);
}

MICKEY_API int grain_set_stream(grain_streams *s, void *cuda_stream) {
  if (!s) return grain_fail(MICKEY_E_ARG, "NULL handle");
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  return set_error(MICKEY_OK, "");
}

MICKEY_API int grain_sync(grain_streams *s) {
  if (!s) return grain_fail(MICKEY_E_ARG, "NULL handle");
  if (cudaStreamSynchronize(s->stream) != cudaSuccess)
    return grain_fail(MICKEY_E_CUDA, "cudaStreamSynchronize");
  return set_error(MICKEY_OK, "");
}

MICKEY_API uint64_t grain_position(const grain_streams *s) { return s ? s->pos : UINT64_MAX; }

MICKEY_API int grain_export_state(grain_streams *s, uint8_t *states) {
  if (!s || !states) return grain_fail(MICKEY_E_ARG, "NULL argument");
  std::vector<uint32_t> w(size_t(2 * kG) * s->Gpad);
  if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
      cudaMemcpy(w.data(), s->d_state, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return grain_fail(MICKEY_E_CUDA, "state copy");
  for (size_t i = 0; i < s->n; ++i) {
    const size_t g = i / 32, l = i % 32;
    uint8_t *rec = states + 20 * i;
    std::memset(rec, 0, 20);
    for (int k = 0; k < 2 * kG; ++k)
      if ((w[size_t(k) * s->Gpad + g] >> l) & 1u) rec[k / 8] |= uint8_t(1u << (k % 8));
  }
  return set_error(MICKEY_OK, "");
}

MICKEY_API int grain_ops_per_clock(int init) { return init ? kGrainInitOps : kGrainOps; }

MICKEY_API void grain_free(grain_streams *s) { grain_release(s); }

}  // extern "C"
