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
#include "keystream_device.cuh"

namespace mickey {
namespace {

// Grid mode: one thread per group, all tiles; rows staged ST tiles deep.
template <int LAYOUT, int U, int ST>
__global__ void __launch_bounds__(kKsThreads)
    keystream_kernel(KeystreamArgs a, EmitCtx e) {
  extern __shared__ uint32_t zs[];
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  run_piece<LAYOUT, U, ST>(a, e, g, zs + threadIdx.x, zs + 32 * kKsThreads + threadIdx.x,
                           zs + kTileBufWords + ST * threadIdx.x, 0,
                           uint32_t((a.n_bits + 31) >> 5));
}

template <int LAYOUT, int U, int ST>
cudaError_t launch_grid_st(const KeystreamArgs &a, const EmitCtx &e, cudaStream_t st) {
  const uint32_t blocks = (a.G + kKsThreads - 1) / kKsThreads;
  const cudaError_t err = allow_smem(keystream_kernel<LAYOUT, U, ST>, ST);
  if (err != cudaSuccess) return err;
  keystream_kernel<LAYOUT, U, ST><<<blocks, kKsThreads, smem_bytes(e, ST), st>>>(a, e);
  return cudaGetLastError();
}

template <int LAYOUT>
cudaError_t launch_grid(const KeystreamArgs &a, int unroll, int depth, const EmitCtx &e,
                        cudaStream_t st) {
  if (unroll != 2 && unroll != 4) return cudaErrorInvalidValue;
  if (depth == 2)
    return unroll == 2 ? launch_grid_st<LAYOUT, 2, 2>(a, e, st) : launch_grid_st<LAYOUT, 4, 2>(a, e, st);
  return unroll == 2 ? launch_grid_st<LAYOUT, 2, 4>(a, e, st) : launch_grid_st<LAYOUT, 4, 4>(a, e, st);
}

}  // namespace

cudaError_t launch_keystream(const KeystreamArgs &a, int layout, int unroll, int stage,
                             const PersistArgs *p, cudaStream_t st) {
  EmitCtx e;
  const uint32_t tail = uint32_t(a.n & 31u);
  e.lane_mask = tail ? ((1u << tail) - 1u) : ~0u;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(a.out);
  e.vec_ok = (addr % 16 == 0) && (a.n_bits % 4 == 0);
  e.word_ok = (addr % 4 == 0) && (((a.n_bits + 7) / 8) % 4 == 0);
  // staging depth: the persistent kernels' own, else 2 or 4 tiles (grid)
  const int depth = p ? int(p->stage_tiles) : (stage == 2 ? 2 : 4);
  e.stage = stage > 0 && layout != MICKEY_LAYOUT_BITSLICED_U32 && (addr % 16 == 0) &&
            (a.n_bits % (32 * uint64_t(depth)) == 0);
  if (p) {
    if (!p->paired) return p->stage_tiles == 4 ? launch_persistent4(a, layout, unroll, e, *p, st)
                                               : cudaErrorInvalidValue;
    switch (p->stage_tiles) {
      case 8: return launch_persistent8(a, layout, unroll, e, *p, st);
      case 4: return launch_paired4(a, layout, unroll, e, *p, st);
      case 2: return launch_paired2(a, layout, unroll, e, *p, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32:
      return launch_grid<MICKEY_LAYOUT_BITSLICED_U32>(a, unroll, depth, e, st);
    case MICKEY_LAYOUT_BYTES:
      return launch_grid<MICKEY_LAYOUT_BYTES>(a, unroll, depth, e, st);
    case MICKEY_LAYOUT_U32:
      return launch_grid<MICKEY_LAYOUT_U32>(a, unroll, depth, e, st);
    case MICKEY_LAYOUT_U32_F32:
      return launch_grid<MICKEY_LAYOUT_U32_F32>(a, unroll, depth, e, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mickey
