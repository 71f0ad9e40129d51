// Device code shared by the keystream launches (grid kernel, persistent
// kernels): emission of 32-clock tiles and run_piece, which clocks one
// group over a range of tiles of the call.
#pragma once

#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "internal.h"

namespace mickey {

struct EmitCtx {
  uint32_t lane_mask;  // valid lanes of this group (last group may be partial)
  bool vec_ok;         // 16-byte vector stores allowed (bitsliced layout)
  bool word_ok;        // 4-byte row stores allowed (bytes layout)
  bool stage;          // row layouts: stage ST tiles per row (8-, 16- or 32-byte stores)
};

// Launches of the persistent kernels (keystream_persistent.cuh), one
// translation unit per kernel and staging depth: the paired clock/emission
// kernel with ST = 8, 4 or 2 tiles (one block per SM), and the two-block
// kernel with ST = 4.
cudaError_t launch_persistent8(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                               const PersistArgs &p, cudaStream_t st);
cudaError_t launch_paired4(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                           const PersistArgs &p, cudaStream_t st);
cudaError_t launch_paired2(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                           const PersistArgs &p, cudaStream_t st);
cudaError_t launch_persistent4(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                               const PersistArgs &p, cudaStream_t st);

namespace {

// Shared memory of a keystream block: two tile buffers (32 words per
// thread each) and, when rows are staged, ST words per row per thread laid
// out [row][thread][ST].  ST = 8 tiles (one block per SM: 160 KiB) writes
// whole 32-byte sectors, so that no partially written sector has to be
// merged in L2 or re-read from DRAM; ST = 4 tiles (16-byte row stores,
// 96 KiB) leaves room for two blocks per SM (the grid kernel and the
// two-block persistent launch).
constexpr size_t kTileBufWords = 2 * 32 * kKsThreads;
constexpr size_t row_stage_words(int st) { return size_t(32) * kKsThreads * st; }

// Store lane l's 32 keystream bits t0..t0+nb-1.  `word` holds z_{t0} in bit
// 31, except for the bytes layout, where it arrives byte-reversed (z_{t0} in
// bit 7, i.e. in memory byte order).  `tile` points at row 32g, column t0 of
// the output; rows are `pitch` bytes apart.
template <int LAYOUT>
__device__ __forceinline__ void store_row_word(uint8_t *tile, uint32_t pitch,
                                               uint64_t f32_off, int l, int nb,
                                               const EmitCtx &e, uint32_t word) {
  uint8_t *o = tile + uint64_t(uint32_t(l) * pitch);
  if constexpr (LAYOUT == MICKEY_LAYOUT_BYTES) {
    if (nb == 32 && e.word_ok) {
      *reinterpret_cast<uint32_t *>(o) = word;
    } else {
      const int nbytes = (nb + 7) >> 3;
      for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(word >> (8 * b));
    }
  } else {
    *reinterpret_cast<uint32_t *>(o) = word;
    if constexpr (LAYOUT == MICKEY_LAYOUT_U32_F32)
      *reinterpret_cast<float *>(o + f32_off) = __uint2float_rn(word >> 8) * 0x1p-24f;
  }
}

// One eighth of the emission of a 32-clock tile held in shared memory
// (column `z`, stride kKsThreads).  Slices must run in order 0..7:
//   bitsliced  slice j stores words 4j..4j+3 (one 128-bit store);
//   row-major  slices 0-3 apply the block swaps of size 4, 2, 1 to rows
//              8j..8j+7 in place; slices 4-7 apply the swaps of size 16 and 8
//              to rows {k, k+8, k+16, k+24} for k = 2(j-4), 2(j-4)+1 and
//              store the finished words.  The five swaps commute, so the
//              result is transpose32() of the tile.
template <int LAYOUT, int ST>
__device__ __forceinline__ void emit_slice(uint32_t *z, uint32_t *rb, const KeystreamArgs &a,
                                           uint32_t g, uint64_t t0, int nb,
                                           const EmitCtx &e, int j) {
  if constexpr (LAYOUT == MICKEY_LAYOUT_BITSLICED_U32) {
    uint32_t *o = static_cast<uint32_t *>(a.out) + size_t(g) * a.n_bits + t0;
    if (nb == 32 && e.vec_ok) {
      uint4 v;
      v.x = z[(4 * j + 0) * kKsThreads] & e.lane_mask;
      v.y = z[(4 * j + 1) * kKsThreads] & e.lane_mask;
      v.z = z[(4 * j + 2) * kKsThreads] & e.lane_mask;
      v.w = z[(4 * j + 3) * kKsThreads] & e.lane_mask;
      reinterpret_cast<uint4 *>(o)[j] = v;
    } else {
      for (int c = 4 * j; c < 4 * j + 4 && c < nb; ++c) o[c] = z[c * kKsThreads] & e.lane_mask;
    }
  } else if (j < 4) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = z[(8 * j + k) * kKsThreads];
    swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
    swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
    swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
    swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
    swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
    swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) z[(8 * j + k) * kKsThreads] = v[k];
  } else {
    const uint32_t pitch = LAYOUT == MICKEY_LAYOUT_BYTES ? uint32_t((a.n_bits + 7) >> 3)
                                                         : uint32_t(a.n_bits >> 3);
    uint8_t *tile = static_cast<uint8_t *>(a.out) + 32ull * g * pitch + (t0 >> 3);
    const uint64_t f32_off = uint64_t(pitch) * a.n;  // float block follows
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * (j - 4) + h;
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = z[(k + 8 * q) * kKsThreads];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes<LAYOUT == MICKEY_LAYOUT_BYTES>(v[0], v[1]);
      swap_bytes<LAYOUT == MICKEY_LAYOUT_BYTES>(v[2], v[3]);
      // row k + 8q of the transposed tile is lane 31 - k - 8q
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = 31 - k - 8 * q;
        if (e.stage && nb == 32)
          rb[l * (kKsThreads * ST) + ((t0 >> 5) & (ST - 1))] = v[q];
        else if ((e.lane_mask >> l) & 1u)
          store_row_word<LAYOUT>(tile, pitch, f32_off, l, nb, e, v[q]);
      }
    }
  }
}

template <int LAYOUT, int ST>
__device__ __forceinline__ void emit_tile(uint32_t *z, uint32_t *rb, const KeystreamArgs &a,
                                          uint32_t g, uint64_t t0, int nb, const EmitCtx &e) {
#pragma unroll 1
  for (int j = 0; j < 8; ++j) emit_slice<LAYOUT, ST>(z, rb, a, g, t0, nb, e, j);
}

// Row layouts with staging: write the staged words of tiles tA..tB (one
// aligned block of ST tiles, or part of one) of every valid row; a whole
// block goes out as ST/4 16-byte stores per row (one 8-byte store for
// ST = 2), and the same for the f32 row.
template <int LAYOUT, int ST>
__device__ __forceinline__ void flush_rows(const uint32_t *rb, const KeystreamArgs &a,
                                           uint32_t g, uint32_t tA, uint32_t tB,
                                           const EmitCtx &e) {
  const uint32_t pitch = uint32_t(a.n_bits >> 3);
  uint8_t *base = static_cast<uint8_t *>(a.out) + 32ull * g * pitch + uint64_t(tA) * 4;
  const uint64_t f32_off = uint64_t(pitch) * a.n;
  const int n = int(tB - tA) + 1, j0 = int(tA & (ST - 1));
#pragma unroll 1
  for (int l = 0; l < 32; ++l) {
    if (!((e.lane_mask >> l) & 1u)) continue;
    const uint32_t *src = rb + l * (kKsThreads * ST);
    uint8_t *o = base + uint64_t(uint32_t(l) * pitch);
    if (ST == 2 && n == ST) {
      const uint2 v = *reinterpret_cast<const uint2 *>(src);
      *reinterpret_cast<uint2 *>(o) = v;
      if constexpr (LAYOUT == MICKEY_LAYOUT_U32_F32) {
        float2 f;
        f.x = __uint2float_rn(v.x >> 8) * 0x1p-24f;
        f.y = __uint2float_rn(v.y >> 8) * 0x1p-24f;
        *reinterpret_cast<float2 *>(o + f32_off) = f;
      }
    } else if (n == ST) {
#pragma unroll
      for (int h = 0; h < ST / 4; ++h) {
        const uint4 v = reinterpret_cast<const uint4 *>(src)[h];
        reinterpret_cast<uint4 *>(o)[h] = v;
        if constexpr (LAYOUT == MICKEY_LAYOUT_U32_F32) {
          float4 f;
          f.x = __uint2float_rn(v.x >> 8) * 0x1p-24f;
          f.y = __uint2float_rn(v.y >> 8) * 0x1p-24f;
          f.z = __uint2float_rn(v.z >> 8) * 0x1p-24f;
          f.w = __uint2float_rn(v.w >> 8) * 0x1p-24f;
          reinterpret_cast<float4 *>(o + f32_off)[h] = f;
        }
      }
    } else {
      for (int j = 0; j < n; ++j) {
        const uint32_t w = src[j0 + j];
        reinterpret_cast<uint32_t *>(o)[j] = w;
        if constexpr (LAYOUT == MICKEY_LAYOUT_U32_F32)
          reinterpret_cast<float *>(o + f32_off)[j] = __uint2float_rn(w >> 8) * 0x1p-24f;
      }
    }
  }
}

// Keystream bits of tiles [tile_a, tile_b) of group g (tile t covers clocks
// 32t .. 32t+31 of this call; the last tile may be partial), continuing from
// and writing back the group's state.  The tile buffer is double-buffered:
// while the 32 clocks of tile k run (U clocks per step), the eight emission
// slices of tile k-1 are interleaved with them, so the clock's independent
// LOP3s hide the latency of the emission's shared-memory and global accesses.
template <int LAYOUT, int U, int ST>
__device__ __forceinline__ void run_piece(const KeystreamArgs &a, EmitCtx e, uint32_t g,
                                          uint32_t *zbuf0, uint32_t *zbuf1, uint32_t *rb,
                                          uint32_t tile_a, uint32_t tile_b) {
  static_assert(U == 2 || U == 4, "one emission slice per 4 clocks");
  const size_t P = a.Gpad;
  uint32_t r[kReg], s[kReg];
  const uint32_t *src = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    r[i] = src[size_t(i) * P];
    s[i] = src[size_t(kReg + i) * P];
  }
  if (g != a.G - 1) e.lane_mask = ~0u;

  const uint32_t full = uint32_t(a.n_bits >> 5);
  const uint32_t fend = tile_b < full ? tile_b : full;
#pragma unroll 1
  for (uint32_t tile = tile_a; tile < fend; ++tile) {
    uint32_t *cur = (tile & 1) ? zbuf1 : zbuf0;
    uint32_t *prev = (tile & 1) ? zbuf0 : zbuf1;
#pragma unroll 1
    for (int c = 0; c < 32; c += U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cur[(c + u) * kKsThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      }
      if (tile > tile_a && (c & 3) == 0)
        emit_slice<LAYOUT, ST>(prev, rb, a, g, uint64_t(tile - 1) << 5, 32, e, c >> 2);
    }
    if (LAYOUT != MICKEY_LAYOUT_BITSLICED_U32 && e.stage && tile > tile_a &&
        ((tile - 1) & (ST - 1)) == ST - 1)
      flush_rows<LAYOUT, ST>(rb, a, g, max(tile - ST, tile_a), tile - 1, e);
  }
  if (fend > tile_a) {
    emit_tile<LAYOUT, ST>((fend & 1) ? zbuf0 : zbuf1, rb, a, g, uint64_t(fend - 1) << 5, 32, e);
    if (LAYOUT != MICKEY_LAYOUT_BITSLICED_U32 && e.stage)
      flush_rows<LAYOUT, ST>(rb, a, g, max((fend - 1) & ~uint32_t(ST - 1), tile_a), fend - 1, e);
  }
  if (tile_b > full && (a.n_bits & 31)) {  // the partial last tile
    uint32_t *cur = (full & 1) ? zbuf1 : zbuf0;
    const int rem = int(a.n_bits & 31);
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
      if (c < rem) {
        cur[c * kKsThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      } else {
        cur[c * kKsThreads] = 0u;
      }
    }
    emit_tile<LAYOUT, ST>(cur, rb, a, g, uint64_t(full) << 5, rem, e);
  }

  uint32_t *dst = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    dst[size_t(i) * P] = r[i];
    dst[size_t(kReg + i) * P] = s[i];
  }
}

size_t smem_bytes(const EmitCtx &e, int st) {
  return 4 * (kTileBufWords + (e.stage ? row_stage_words(st) : 0));
}

template <class K>
cudaError_t allow_smem(K kernel, int st) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(4 * (kTileBufWords + row_stage_words(st))));
}

}  // namespace
}  // namespace mickey
