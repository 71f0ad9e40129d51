// Persistent keystream kernel: equal segments of the groups x tiles work
// line per warp, with a bounded hand-off of the state between segments.
// Included by one translation unit per staging depth ST.
#pragma once

#include "keystream_device.cuh"

namespace mickey {
namespace {

__device__ __forceinline__ uint32_t load_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void store_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Piece k (in processing order) of the work-line segment of warp `slot`:
// warp-group w, tiles [ta, tb).  Returns false past the last piece.  The
// order is: the head of the last warp-group (if the segment ends inside it),
// the whole warp-groups, the tail of the first warp-group (if the segment
// starts inside it).  Recomputed per piece so that only (slot, k) stay live
// across the clock loop.
__device__ __forceinline__ bool segment_piece(const PersistArgs &p, uint64_t NT, uint32_t slot,
                                              uint32_t k, uint32_t &w, uint32_t &ta,
                                              uint32_t &tb) {
  const uint64_t total = uint64_t(p.W) * NT;
  const uint64_t seg_a = uint64_t(slot) * p.L;
  const uint64_t seg_b = seg_a + p.L < total ? seg_a + p.L : total;
  if (seg_a >= seg_b) return false;
  const uint64_t w_first = seg_a / NT, w_last = (seg_b - 1) / NT;
  const bool has_tail = seg_a > w_first * NT;
  const bool has_head = (seg_b - w_last * NT) < NT && !(has_tail && w_last == w_first);
  const uint64_t full_lo = w_first + (has_tail ? 1 : 0);
  const uint64_t full_end = w_last + 1 - (has_head ? 1 : 0);
  const uint64_t full_n = full_end > full_lo ? full_end - full_lo : 0;
  const uint64_t n_pieces = (has_head ? 1 : 0) + full_n + (has_tail ? 1 : 0);
  if (k >= n_pieces) return false;
  const uint64_t kk = k - (has_head ? 1 : 0);
  const uint64_t ww = (has_head && k == 0) ? w_last : (kk < full_n ? full_lo + kk : w_first);
  w = uint32_t(ww);
  ta = uint32_t(ww == w_first ? seg_a - ww * NT : 0);
  tb = uint32_t(ww == w_last ? seg_b - ww * NT : NT);
  return true;
}

// Persistent mode with two blocks per SM (ST = 4): two warps per SM
// sub-partition, each clocking and emitting its own tiles, launched
// cooperatively (all warps resident).  The work line -- warp-group w (32 groups) x tile t,
// W x NT tiles in all -- is cut into equal segments, one per warp, so every
// sub-partition gets the same work even when W is not a multiple of the
// warp count.  A segment holds at most one piece of the warp-group it
// starts in (a tail: tiles ta..NT) and one of the group it ends in (a head:
// tiles 0..tb).  A warp runs its head piece first and publishes the state,
// then its whole groups, then its tail piece, which continues from the
// state the previous segment's head published (bounded acquire-spin; on
// timeout the error flag is raised and the piece is skipped).
template <int LAYOUT, int U, int ST>
__global__ void __launch_bounds__(kKsThreads, 8 / ST)
    keystream_persistent_kernel(KeystreamArgs a, EmitCtx e, PersistArgs p) {
  extern __shared__ uint32_t zs[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t slot = blockIdx.x * (kKsThreads / 32) + (threadIdx.x >> 5);
  const uint64_t NT = (a.n_bits + 31) >> 5;
#pragma unroll 1
  for (uint32_t k = 0;; ++k) {
    uint32_t w, ta, tb;
    if (!segment_piece(p, NT, slot, k, w, ta, tb)) break;
    if (ta > 0) {  // tail: wait for the head piece of this warp-group
      uint32_t it = 0;
      bool ok = true;
      while (load_acquire(p.flags + w) != p.wait_epoch) {
        if (++it > p.spin_limit) {
          ok = false;
          break;
        }
        __nanosleep(256);
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(p.err, kErrTimeout);
        continue;
      }
    }
    const uint32_t g = w * 32 + lane;
    if (g < a.G)
      run_piece<LAYOUT, U, ST>(a, e, g, zs + threadIdx.x, zs + 32 * kKsThreads + threadIdx.x,
                               zs + kTileBufWords + ST * threadIdx.x, ta, tb);
    if (ta == 0 && tb < NT) {  // head: publish the state for the next segment
      __threadfence();
      __syncwarp();
      if (lane == 0) store_release(p.flags + w, p.epoch);
    }
  }
}

// Rendezvous of the clock warp and the emission warp of pair `id` (1..4):
// a named barrier of 64 threads.  The non-aligned form lets the lanes of a
// warp arrive from divergent code.
__device__ __forceinline__ void pair_sync(uint32_t id) {
  asm volatile("barrier.sync %0, 64;" ::"r"(id) : "memory");
}

// Clock side of a piece (warp-specialised launch): the 32 clocks of each
// tile write their z words into the tile buffer of parity `par`, then the
// pair meets; the emission warp takes that buffer while the next tile is
// clocked into the other one.  Lanes past the last group clock a zero state
// and write nothing to global memory, but meet at every barrier.
template <int U>
__device__ __forceinline__ void clock_piece(const KeystreamArgs &a, uint32_t g, uint32_t *zb0,
                                            uint32_t *zb1, uint32_t &par, uint32_t bar,
                                            uint32_t tile_a, uint32_t tile_b) {
  const size_t P = a.Gpad;
  const bool valid = g < a.G;
  uint32_t r[kReg], s[kReg];
  const uint32_t *src = a.state + (valid ? g : 0);
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    r[i] = valid ? src[size_t(i) * P] : 0u;
    s[i] = valid ? src[size_t(kReg + i) * P] : 0u;
  }
  const uint32_t full = uint32_t(a.n_bits >> 5);
  const uint32_t fend = tile_b < full ? tile_b : full;
#pragma unroll 1
  for (uint32_t tile = tile_a; tile < fend; ++tile) {
    uint32_t *cur = par ? zb1 : zb0;
#pragma unroll 1
    for (int c = 0; c < 32; c += U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cur[(c + u) * kKsThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      }
    }
    pair_sync(bar);
    par ^= 1u;
  }
  if (tile_b > full && (a.n_bits & 31)) {  // the partial last tile
    uint32_t *cur = par ? zb1 : zb0;
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
    pair_sync(bar);
    par ^= 1u;
  }
  if (valid) {
    uint32_t *dst = a.state + g;
#pragma unroll
    for (int i = 0; i < kReg; ++i) {
      dst[size_t(i) * P] = r[i];
      dst[size_t(kReg + i) * P] = s[i];
    }
  }
}

// Emission side of the same piece: after each rendezvous, un-bitslice and
// store the tile the clock warp has just finished, and write out the staged
// rows at the end of every aligned block of ST tiles and at the end of the
// piece.  Meets the clock warp exactly as often as clock_piece does.
template <int LAYOUT, int ST>
__device__ __forceinline__ void emit_piece(const KeystreamArgs &a, EmitCtx e, uint32_t g,
                                           uint32_t *zb0, uint32_t *zb1, uint32_t *rb,
                                           uint32_t &par, uint32_t bar, uint32_t tile_a,
                                           uint32_t tile_b) {
  const bool valid = g < a.G;
  if (g != a.G - 1) e.lane_mask = ~0u;
  const uint32_t full = uint32_t(a.n_bits >> 5);
  const uint32_t fend = tile_b < full ? tile_b : full;
#pragma unroll 1
  for (uint32_t tile = tile_a; tile < fend; ++tile) {
    pair_sync(bar);
    if (valid) {
      emit_tile<LAYOUT, ST>(par ? zb1 : zb0, rb, a, g, uint64_t(tile) << 5, 32, e);
      if (LAYOUT != MICKEY_LAYOUT_BITSLICED_U32 && e.stage &&
          ((tile & (ST - 1)) == ST - 1 || tile == fend - 1))
        flush_rows<LAYOUT, ST>(rb, a, g, max(tile & ~uint32_t(ST - 1), tile_a), tile, e);
    }
    par ^= 1u;
  }
  if (tile_b > full && (a.n_bits & 31)) {
    pair_sync(bar);
    if (valid)
      emit_tile<LAYOUT, ST>(par ? zb1 : zb0, rb, a, g, uint64_t(full) << 5, int(a.n_bits & 31), e);
    par ^= 1u;
  }
}

// Warp-specialised persistent launch (ST = 8, one block per SM): each SM
// sub-partition runs a clock warp (threads 0..127: the 200 state words and
// nothing else in registers, so the clock issues as densely as it does
// alone) and an emission warp (threads 128..255: transposes and stores).
// Clock warp w and emission warp w + 4 form pair w; they work through the
// same segment of the work line as one warp of keystream_persistent_kernel
// and meet once per tile at named barrier 1 + w, the tile buffers
// alternating between them.  The hand-off of a tail piece is the clock
// warp's; when its wait runs out it raises the error flag and clocks the
// piece anyway, so both warps still meet the same number of times.  With
// fewer warp-groups than clock warps the same kernel runs one whole
// warp-group per pair (L = NT, no pieces to hand off), launched without the
// cooperative attribute.
template <int LAYOUT, int U, int ST>
__global__ void __launch_bounds__(2 * kKsThreads, 1)
    keystream_ws_kernel(KeystreamArgs a, EmitCtx e, PersistArgs p) {
  extern __shared__ uint32_t zs[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t t = threadIdx.x & (kKsThreads - 1);   // thread of the clock side
  const uint32_t pair = t >> 5;
  const bool clocker = threadIdx.x < kKsThreads;
  const uint32_t slot = blockIdx.x * (kKsThreads / 32) + pair;
  const uint64_t NT = (a.n_bits + 31) >> 5;
  uint32_t *zb0 = zs + t, *zb1 = zs + 32 * kKsThreads + t;
  uint32_t par = 0;
#pragma unroll 1
  for (uint32_t k = 0;; ++k) {
    uint32_t w, ta, tb;
    if (!segment_piece(p, NT, slot, k, w, ta, tb)) break;
    const uint32_t g = w * 32 + lane;
    if (clocker) {
      if (ta > 0) {  // tail: wait for the head piece of this warp-group
        uint32_t it = 0;
        bool ok = true;
        while (load_acquire(p.flags + w) != p.wait_epoch) {
          if (++it > p.spin_limit) {
            ok = false;
            break;
          }
          __nanosleep(256);
        }
        if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(p.err, kErrTimeout);
      }
      clock_piece<U>(a, g, zb0, zb1, par, 1 + pair, ta, tb);
      if (ta == 0 && tb < NT) {  // head: publish the state for the next segment
        __threadfence();
        __syncwarp();
        if (lane == 0) store_release(p.flags + w, p.epoch);
      }
    } else {
      emit_piece<LAYOUT, ST>(a, e, g, zb0, zb1, zs + kTileBufWords + ST * t, par, 1 + pair, ta,
                             tb);
    }
  }
}

template <int LAYOUT, int U, int ST>
cudaError_t launch_ws_kernel(const KeystreamArgs &a, const EmitCtx &e, const PersistArgs &p,
                             cudaStream_t st) {
  cudaError_t err = allow_smem(keystream_ws_kernel<LAYOUT, U, ST>, ST);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.dynamicSmemBytes = smem_bytes(e, ST);
  cfg.gridDim = dim3(p.blocks);
  cfg.blockDim = dim3(2 * kKsThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = p.cooperative ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, keystream_ws_kernel<LAYOUT, U, ST>, a, e, p);
}

template <int LAYOUT, int U, int ST>
cudaError_t launch_persistent_kernel(const KeystreamArgs &a, const EmitCtx &e,
                                     const PersistArgs &p, cudaStream_t st) {
  cudaError_t err = allow_smem(keystream_persistent_kernel<LAYOUT, U, ST>, ST);
  if (err != cudaSuccess) return err;
  cudaLaunchConfig_t cfg = {};
  cfg.dynamicSmemBytes = smem_bytes(e, ST);
  cfg.gridDim = dim3(p.blocks);
  cfg.blockDim = dim3(kKsThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, keystream_persistent_kernel<LAYOUT, U, ST>, a, e, p);
}

template <int LAYOUT, int ST>
cudaError_t launch_ws_unroll(const KeystreamArgs &a, int unroll, const EmitCtx &e,
                             const PersistArgs &p, cudaStream_t st) {
  switch (unroll) {
    case 2: return launch_ws_kernel<LAYOUT, 2, ST>(a, e, p, st);
    case 4: return launch_ws_kernel<LAYOUT, 4, ST>(a, e, p, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int ST>
cudaError_t launch_ws_st(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                         const PersistArgs &p, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32:
      err = launch_ws_unroll<MICKEY_LAYOUT_BITSLICED_U32, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_BYTES:
      err = launch_ws_unroll<MICKEY_LAYOUT_BYTES, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_U32:
      err = launch_ws_unroll<MICKEY_LAYOUT_U32, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_U32_F32:
      err = launch_ws_unroll<MICKEY_LAYOUT_U32_F32, ST>(a, unroll, e, p, st);
      break;
    default: break;
  }
  return err != cudaSuccess ? err : cudaGetLastError();
}

template <int LAYOUT, int ST>
cudaError_t launch_persistent_unroll(const KeystreamArgs &a, int unroll, const EmitCtx &e,
                                     const PersistArgs &p, cudaStream_t st) {
  switch (unroll) {
    case 2: return launch_persistent_kernel<LAYOUT, 2, ST>(a, e, p, st);
    case 4: return launch_persistent_kernel<LAYOUT, 4, ST>(a, e, p, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int ST>
cudaError_t launch_persistent_st(const KeystreamArgs &a, int layout, int unroll,
                                 const EmitCtx &e, const PersistArgs &p, cudaStream_t st) {
  cudaError_t err = cudaErrorInvalidValue;
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32:
      err = launch_persistent_unroll<MICKEY_LAYOUT_BITSLICED_U32, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_BYTES:
      err = launch_persistent_unroll<MICKEY_LAYOUT_BYTES, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_U32:
      err = launch_persistent_unroll<MICKEY_LAYOUT_U32, ST>(a, unroll, e, p, st);
      break;
    case MICKEY_LAYOUT_U32_F32:
      err = launch_persistent_unroll<MICKEY_LAYOUT_U32_F32, ST>(a, unroll, e, p, st);
      break;
    default: break;
  }
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace
}  // namespace mickey
