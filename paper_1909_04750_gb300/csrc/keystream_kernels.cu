// Bitsliced MICKEY 2.0 keystream generation (Sec. IV-D) with the output
// written in one of four layouts.
//
// One thread owns one 32-lane group: its 200 state words stay in registers
// for the whole call.  Each clock produces z = r0 ^ s0 (one word = one
// keystream bit of 32 instances) and then runs one non-mixing CLOCK_KG.
// Words are staged in shared memory (one column per thread, conflict-free)
// and every 32 clocks the tile is emitted:
//   bitsliced  the 32 words as they are, eight 128-bit stores;
//   row-major  a 32x32 bit-matrix transpose turns the tile into one 32-bit
//              word per instance (the un-bitslicing of Sec. IV-A run
//              backwards), stored as bytes, big-endian u32, or u32 + FP32.
// Finally the state is written back so the next call continues the streams.
#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "internal.h"

namespace mickey {
namespace {

struct EmitCtx {
  uint32_t lane_mask;  // valid lanes of this group (last group may be partial)
  bool vec_ok;         // 16-byte vector stores allowed (bitsliced layout)
  bool word_ok;        // 4-byte row stores allowed (bytes layout)
};

template <int J>
__device__ __forceinline__ void swap_bits(uint32_t &lo, uint32_t &hi) {
  constexpr uint32_t m = J == 4 ? 0x0F0F0F0Fu : J == 2 ? 0x33333333u : 0x55555555u;
  const uint32_t t = (lo ^ (hi >> J)) & m;
  lo ^= t;
  hi ^= t << J;
}
// Block swap of size 16: lo keeps its high half and takes hi's high half;
// hi keeps its low half and takes lo's low half.
__device__ __forceinline__ void swap_halves(uint32_t &lo, uint32_t &hi) {
  const uint32_t a = __byte_perm(lo, hi, 0x3276);
  hi = __byte_perm(lo, hi, 0x1054);
  lo = a;
}
// Block swap of size 8 (bytes 1 and 3 of hi into bytes 0 and 2 of lo and
// bytes 0 and 2 of lo into bytes 1 and 3 of hi).
__device__ __forceinline__ void swap_bytes(uint32_t &lo, uint32_t &hi) {
  const uint32_t a = __byte_perm(lo, hi, 0x3715);
  hi = __byte_perm(lo, hi, 0x2604);
  lo = a;
}

// Store lane l's 32 keystream bits t0..t0+nb-1 (z_{t0} in bit 31).  `tile`
// points at row 32g, column t0 of the output; rows are `pitch` bytes apart.
template <int LAYOUT>
__device__ __forceinline__ void store_row_word(uint8_t *tile, uint32_t pitch,
                                               uint64_t f32_off, int l, int nb,
                                               const EmitCtx &e, uint32_t word) {
  uint8_t *o = tile + uint64_t(uint32_t(l) * pitch);
  if constexpr (LAYOUT == MICKEY_LAYOUT_BYTES) {
    if (nb == 32 && e.word_ok) {
      *reinterpret_cast<uint32_t *>(o) = __byte_perm(word, 0u, 0x0123);
    } else {
      const int nbytes = (nb + 7) >> 3;
      for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(word >> (24 - 8 * b));
    }
  } else {
    *reinterpret_cast<uint32_t *>(o) = word;
    if constexpr (LAYOUT == MICKEY_LAYOUT_U32_F32)
      *reinterpret_cast<float *>(o + f32_off) = __uint2float_rn(word >> 8) * 0x1p-24f;
  }
}

template <int LAYOUT>
__device__ __forceinline__ void emit_tile(const uint32_t *zcol,
                                          const KeystreamArgs &a, uint32_t g,
                                          uint64_t t0, int nb,
                                          const EmitCtx &e) {
  if constexpr (LAYOUT == MICKEY_LAYOUT_BITSLICED_U32) {
    uint32_t *o = static_cast<uint32_t *>(a.out) + size_t(g) * a.n_bits + t0;
    if (nb == 32 && e.vec_ok) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint4 v;
        v.x = zcol[(4 * q + 0) * kKsThreads] & e.lane_mask;
        v.y = zcol[(4 * q + 1) * kKsThreads] & e.lane_mask;
        v.z = zcol[(4 * q + 2) * kKsThreads] & e.lane_mask;
        v.w = zcol[(4 * q + 3) * kKsThreads] & e.lane_mask;
        reinterpret_cast<uint4 *>(o)[q] = v;
      }
    } else {
      for (int c = 0; c < nb; ++c) o[c] = zcol[c * kKsThreads] & e.lane_mask;
    }
  } else {
    // Un-bitslice the 32x32 tile in two passes over shared memory, eight or
    // four words live at a time: the block swaps of size 4, 2, 1 act within
    // 8-row chunks and those of size 16, 8 within the rows {k, k+8, k+16,
    // k+24}; the five swaps commute, so this equals transpose32().
    uint32_t *z = const_cast<uint32_t *>(zcol);
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = z[(8 * c + k) * kKsThreads];
      swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
      swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
      swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
      swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
      swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
      swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
      for (int k = 0; k < 8; ++k) z[(8 * c + k) * kKsThreads] = v[k];
    }
    const uint32_t pitch = LAYOUT == MICKEY_LAYOUT_BYTES ? uint32_t((a.n_bits + 7) >> 3)
                                                         : uint32_t(a.n_bits >> 3);
    uint8_t *tile = static_cast<uint8_t *>(a.out) + 32ull * g * pitch + (t0 >> 3);
    const uint64_t f32_off = uint64_t(pitch) * a.n;  // float block follows
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = z[(k + 8 * q) * kKsThreads];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes(v[0], v[1]);
      swap_bytes(v[2], v[3]);
      // row k + 8q of the transposed tile is lane 31 - k - 8q
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = 31 - k - 8 * q;
        if ((e.lane_mask >> l) & 1u) store_row_word<LAYOUT>(tile, pitch, f32_off, l, nb, e, v[q]);
      }
    }
  }
}

template <int LAYOUT, int U>
__global__ void __launch_bounds__(kKsThreads)
    keystream_kernel(KeystreamArgs a, EmitCtx e) {
  __shared__ uint32_t zs[32 * kKsThreads];
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  const size_t P = a.Gpad;

  uint32_t r[kReg], s[kReg];
  const uint32_t *src = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    r[i] = src[size_t(i) * P];
    s[i] = src[size_t(kReg + i) * P];
  }
  if (g != a.G - 1) e.lane_mask = ~0u;

  uint32_t *zcol = zs + threadIdx.x;
  const uint64_t full_end = a.n_bits & ~uint64_t(31);
  uint64_t t0 = 0;
#pragma unroll 1
  for (; t0 < full_end; t0 += 32) {
#pragma unroll 1
    for (int c = 0; c < 32; c += U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        zcol[(c + u) * kKsThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      }
    }
    emit_tile<LAYOUT>(zcol, a, g, t0, 32, e);
  }
  if (t0 < a.n_bits) {
    const int rem = int(a.n_bits - t0);
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
      if (c < rem) {
        zcol[c * kKsThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      } else {
        zcol[c * kKsThreads] = 0u;
      }
    }
    emit_tile<LAYOUT>(zcol, a, g, t0, rem, e);
  }

  uint32_t *dst = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    dst[size_t(i) * P] = r[i];
    dst[size_t(kReg + i) * P] = s[i];
  }
}

template <int LAYOUT>
cudaError_t launch_layout(const KeystreamArgs &a, int unroll, const EmitCtx &e,
                          cudaStream_t st) {
  const uint32_t blocks = (a.G + kKsThreads - 1) / kKsThreads;
  switch (unroll) {
    case 2: keystream_kernel<LAYOUT, 2><<<blocks, kKsThreads, 0, st>>>(a, e); break;
    case 4: keystream_kernel<LAYOUT, 4><<<blocks, kKsThreads, 0, st>>>(a, e); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_keystream(const KeystreamArgs &a, int layout, int unroll,
                             cudaStream_t st) {
  EmitCtx e;
  const uint32_t tail = uint32_t(a.n & 31u);
  e.lane_mask = tail ? ((1u << tail) - 1u) : ~0u;
  const uintptr_t p = reinterpret_cast<uintptr_t>(a.out);
  e.vec_ok = (p % 16 == 0) && (a.n_bits % 4 == 0);
  e.word_ok = (p % 4 == 0) && (((a.n_bits + 7) / 8) % 4 == 0);
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32:
      return launch_layout<MICKEY_LAYOUT_BITSLICED_U32>(a, unroll, e, st);
    case MICKEY_LAYOUT_BYTES:
      return launch_layout<MICKEY_LAYOUT_BYTES>(a, unroll, e, st);
    case MICKEY_LAYOUT_U32:
      return launch_layout<MICKEY_LAYOUT_U32>(a, unroll, e, st);
    case MICKEY_LAYOUT_U32_F32:
      return launch_layout<MICKEY_LAYOUT_U32_F32>(a, unroll, e, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mickey
