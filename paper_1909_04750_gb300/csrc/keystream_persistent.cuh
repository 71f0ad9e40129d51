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

// Persistent mode: one warp per SM sub-partition (ST = 8, one block per SM)
// or two (ST = 4, two blocks per SM), launched cooperatively (all warps
// resident).  The work line -- warp-group w (32 groups) x tile t,
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
