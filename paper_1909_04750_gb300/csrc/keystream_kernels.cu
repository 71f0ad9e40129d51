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

// Grid mode: one thread per group, all tiles.
template <int LAYOUT, int U>
__global__ void __launch_bounds__(kKsThreads)
    keystream_kernel(KeystreamArgs a, EmitCtx e) {
  extern __shared__ uint32_t zs[];
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  run_piece<LAYOUT, U, 4>(a, e, g, zs + threadIdx.x, zs + 32 * kKsThreads + threadIdx.x,
                          zs + kTileBufWords + 4 * threadIdx.x, 0,
                       uint32_t((a.n_bits + 31) >> 5));
}

template <int LAYOUT>
cudaError_t launch_grid(const KeystreamArgs &a, int unroll, const EmitCtx &e, cudaStream_t st) {
  const uint32_t blocks = (a.G + kKsThreads - 1) / kKsThreads;
  const size_t smem = smem_bytes(e, 4);
  cudaError_t err = cudaSuccess;
  switch (unroll) {
    case 2:
      err = allow_smem(keystream_kernel<LAYOUT, 2>, 4);
      if (err == cudaSuccess) keystream_kernel<LAYOUT, 2><<<blocks, kKsThreads, smem, st>>>(a, e);
      break;
    case 4:
      err = allow_smem(keystream_kernel<LAYOUT, 4>, 4);
      if (err == cudaSuccess) keystream_kernel<LAYOUT, 4><<<blocks, kKsThreads, smem, st>>>(a, e);
      break;
    default: return cudaErrorInvalidValue;
  }
  return err != cudaSuccess ? err : cudaGetLastError();
}

}  // namespace

cudaError_t launch_keystream(const KeystreamArgs &a, int layout, int unroll, bool stage,
                             const PersistArgs *p, cudaStream_t st) {
  EmitCtx e;
  const uint32_t tail = uint32_t(a.n & 31u);
  e.lane_mask = tail ? ((1u << tail) - 1u) : ~0u;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(a.out);
  e.vec_ok = (addr % 16 == 0) && (a.n_bits % 4 == 0);
  e.word_ok = (addr % 4 == 0) && (((a.n_bits + 7) / 8) % 4 == 0);
  e.stage = stage && layout != MICKEY_LAYOUT_BITSLICED_U32 && (addr % 16 == 0) &&
            (a.n_bits % (p ? 32 * p->stage_tiles : 128) == 0);
  if (p) {
    if (p->stage_tiles == 8) return launch_persistent8(a, layout, unroll, e, *p, st);
    if (p->stage_tiles == 4) return launch_persistent4(a, layout, unroll, e, *p, st);
    return cudaErrorInvalidValue;
  }
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32:
      return launch_grid<MICKEY_LAYOUT_BITSLICED_U32>(a, unroll, e, st);
    case MICKEY_LAYOUT_BYTES:
      return launch_grid<MICKEY_LAYOUT_BYTES>(a, unroll, e, st);
    case MICKEY_LAYOUT_U32:
      return launch_grid<MICKEY_LAYOUT_U32>(a, unroll, e, st);
    case MICKEY_LAYOUT_U32_F32:
      return launch_grid<MICKEY_LAYOUT_U32_F32>(a, unroll, e, st);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mickey
