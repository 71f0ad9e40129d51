// Ragged keystream generation on a streams handle: every stream continues
// by its own number of bits in one launch (the instance-per-lane design of
// Sec. IV-D with uneven lengths).
//
// One thread owns one 32-lane group, as in the keystream kernels: the
// group's 200 state words stay in registers and the group is clocked as
// many times as its longest lane needs.  Two things make the lanes' lengths
// differ without a per-clock cost:
//   * the keystream word of a clock is taken as (r0 ^ s0) & alive, one LOP3
//     like the plain XOR, where `alive` holds the lanes whose length has not
//     been reached; the bits of finished lanes are zero, so a row store only
//     has to stop at the row's last byte;
//   * a lane's state must be the one after exactly its own number of clocks.
//     When the group starts, the bits of every lane with a length above 0
//     are cleared in the state in HBM (unless all lanes share one length);
//     at each distinct end point E of the group (at most 32) the current
//     words, masked to the lanes ending at E, are OR-ed in (one fire-and-
//     forget atomic per word, so the clock loop does not wait for memory),
//     or stored outright when those lanes are all the group's lanes.  Lanes
//     asked for 0 bits are never touched.
// The clock loop takes one clock per iteration, so that the write-back code
// exists once: a thread that takes it holds up its warp, and unrolled copies
// of it were instruction-cache misses each time.  The values the next clock
// reads besides neighbouring bits (control bit, feedback bits) are computed
// inside the iteration, so the loop's back edge does not wait on them.  An
// end point is found from a per-tile mask of the clocks at which some lane
// ends; the lanes ending there are looked up only then.  Every fourth clock
// emits one eighth of the previous tile (as the keystream kernels do).  The
// last tile is clocked in full: past the longest lane every lane has been
// written back and the extra keystream bits are zero and not stored.
#include "bitslice.cuh"
#include "internal.h"
#include "../../include/mickey.h"

namespace mickey {
namespace {

constexpr int kRaggedThreads = 64;

// Per-thread view of the group's lanes in shared memory: lane l's length at
// bits[l * kRaggedThreads] and its output row's address at row[l * kRaggedThreads]
// (columns of one thread, so a warp's accesses are conflict-free).
struct LaneTab {
  const uint64_t *bits;
  uint8_t *const *row;
};

// Bit k set when some lane's length is t0 + k + 1 (its last clock is clock
// k of the tile starting at call clock t0).
__device__ __forceinline__ uint32_t tile_ends(const LaneTab &lt, int lanes, uint64_t t0) {
  uint32_t e = 0;
  for (int l = 0; l < lanes; ++l) {
    const uint64_t d = lt.bits[l * kRaggedThreads] - t0 - 1;   // wraps for lengths <= t0
    if (d < 32) e |= 1u << d;
  }
  return e;
}

// The lanes whose length is exactly E.
__device__ __forceinline__ uint32_t lanes_ending(const LaneTab &lt, int lanes, uint64_t E) {
  uint32_t m = 0;
  for (int l = 0; l < lanes; ++l) m |= (lt.bits[l * kRaggedThreads] == E ? 1u : 0u) << l;
  return m;
}

// True when every lane has length C (then the one end point writes the
// whole group back with plain stores).
__device__ __forceinline__ bool same_end(const LaneTab &lt, int lanes, uint64_t C) {
  for (int l = 0; l < lanes; ++l)
    if (lt.bits[l * kRaggedThreads] != C) return false;
  return true;
}

// Truth table of (a ^ b) & c (operands a, b, c = 0xF0, 0xCC, 0xAA).
constexpr uint32_t kXorAnd = ((0xF0u ^ 0xCCu) & 0xAAu) & 0xFFu;              // 0x28

// Merge the lanes in `m` of the current state into the state in HBM
// (`pad`: lanes past the last instance, whose bits nothing reads).  The bits
// of every lane with a length above 0 were cleared in HBM when the group
// started, so setting the ones is enough.  The base address and stride
// pass through an opaque move, so that the 200 word addresses are formed
// here, when the branch is taken, and are not held live across the clock
// loop (which spilled).
__device__ __forceinline__ void snapshot(uint32_t *st0, size_t P0, const uint32_t (&r)[kReg],
                                         const uint32_t (&s)[kReg], uint32_t m, uint32_t pad) {
  uint32_t *st;
  size_t P;
  asm volatile("mov.b64 %0, %1;" : "=l"(st) : "l"(st0));
  asm volatile("mov.b64 %0, %1;" : "=l"(P) : "l"(P0));
  if ((m | pad) == ~0u) {
#pragma unroll
    for (int i = 0; i < kReg; ++i) {
      st[size_t(i) * P] = r[i];
      st[size_t(kReg + i) * P] = s[i];
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    atomicOr(st + size_t(i) * P, r[i] & m);
    atomicOr(st + size_t(kReg + i) * P, s[i] & m);
  }
}

// Store the finished word w of lane l (z_{t0} first; memory byte order for
// the bytes layout, big-endian for u32) of the tile starting at call clock
// t0, up to the lane's last byte.
template <int LAYOUT>
__device__ __forceinline__ void store_lane(const LaneTab &lt, int l, uint64_t t0, uint32_t w) {
  const uint64_t bits = lt.bits[l * kRaggedThreads];
  if (t0 >= bits) return;
  uint8_t *o = lt.row[l * kRaggedThreads] + (t0 >> 3);
  const uint64_t left = bits - t0;
  if (left >= 32 && (reinterpret_cast<uintptr_t>(o) & 3u) == 0) {
    *reinterpret_cast<uint32_t *>(o) = w;
    return;
  }
  // bytes layout only: a last partial word or an unaligned row
  const int nbytes = left >= 32 ? 4 : int((left + 7) >> 3);
  for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(w >> (8 * b));
}

// One eighth of a tile's emission (slices must run in order 0..7).
//   bitsliced  slice j stores words 4j..4j+3 of the group's row;
//   row-major  the two-pass in-place transpose of the keystream kernels:
//              slices 0-3 swap blocks of size 4, 2, 1; slices 4-7 swap blocks
//              of size 16 and 8 and store.
template <int LAYOUT>
__device__ __forceinline__ void ragged_slice(uint32_t *z, const LaneTab &lt, uint8_t *grow,
                                             int lanes, uint64_t t0, int cnt, uint64_t C,
                                             int j) {
  if constexpr (LAYOUT == MICKEY_LAYOUT_BITSLICED_U32) {
    uint32_t *o = reinterpret_cast<uint32_t *>(grow) + t0;
    if (cnt == 32 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
      uint4 v;
      v.x = z[(4 * j + 0) * kRaggedThreads];
      v.y = z[(4 * j + 1) * kRaggedThreads];
      v.z = z[(4 * j + 2) * kRaggedThreads];
      v.w = z[(4 * j + 3) * kRaggedThreads];
      reinterpret_cast<uint4 *>(o)[j] = v;
    } else {
      for (int c = 4 * j; c < 4 * j + 4 && uint64_t(c) < C - t0 && c < cnt; ++c)
        o[c] = z[c * kRaggedThreads];
    }
  } else if (j < 4) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = z[(8 * j + k) * kRaggedThreads];
    swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
    swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
    swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
    swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
    swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
    swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) z[(8 * j + k) * kRaggedThreads] = v[k];
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * (j - 4) + h;
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = z[(k + 8 * q) * kRaggedThreads];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes<LAYOUT == MICKEY_LAYOUT_BYTES>(v[0], v[1]);
      swap_bytes<LAYOUT == MICKEY_LAYOUT_BYTES>(v[2], v[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = 31 - k - 8 * q;   // row k + 8q of the transposed tile
        if (l < lanes) store_lane<LAYOUT>(lt, l, t0, v[q]);
      }
    }
  }
}

template <int LAYOUT>
__device__ __forceinline__ void ragged_tile(uint32_t *z, const LaneTab &lt, uint8_t *grow,
                                            int lanes, uint64_t t0, int cnt, uint64_t C) {
#pragma unroll 1
  for (int j = 0; j < 8; ++j) ragged_slice<LAYOUT>(z, lt, grow, lanes, t0, cnt, C, j);
}

// In-tile index of the clock after which the lanes ending at `next` are done
// (next > t0), or 64 when that end point lies beyond the tile.
__device__ __forceinline__ int end_in_tile(uint64_t next, uint64_t t0) {
  return next - t0 - 1 < 32 ? int(next - t0 - 1) : 64;
}

// Shared memory of a block: two tile buffers (32 words per thread), then the
// lane table: lengths and row addresses, 32 of each per thread.
constexpr size_t kRaggedSmem = (2 * 32 * 4 + 32 * 8 + 32 * 8) * size_t(kRaggedThreads);

template <int LAYOUT>
__global__ void __launch_bounds__(kRaggedThreads) ragged_kernel(RaggedArgs a) {
  extern __shared__ __align__(16) uint32_t zs[];
  uint64_t *tab = reinterpret_cast<uint64_t *>(zs + 2 * 32 * kRaggedThreads);
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.G) return;
  const uint64_t base = uint64_t(g) * 32;
  const int lanes = a.n - base >= 32 ? 32 : int(a.n - base);
  const uint32_t pad = lanes < 32 ? ~0u << lanes : 0u;
  LaneTab lt{tab + threadIdx.x, reinterpret_cast<uint8_t *const *>(tab + 32 * kRaggedThreads +
                                                                    threadIdx.x)};
  uint64_t C = 0;
  uint32_t alive = 0;
  for (int l = 0; l < lanes; ++l) {
    const uint64_t b = a.n_bits[base + l];
    tab[l * kRaggedThreads + threadIdx.x] = b;
    if (LAYOUT != MICKEY_LAYOUT_BITSLICED_U32)
      tab[(32 + l) * kRaggedThreads + threadIdx.x] =
          reinterpret_cast<uint64_t>(a.out + a.offsets[base + l]);
    C = max(C, b);
    alive |= (b > 0 ? 1u : 0u) << l;
  }
  uint8_t *grow = LAYOUT == MICKEY_LAYOUT_BITSLICED_U32 ? a.out + a.offsets[g] : nullptr;
  if (alive == 0) return;                     // every lane asks for 0 bits

  const size_t P = a.Gpad;
  uint32_t *st = a.state + g;
  uint32_t r[kReg], s[kReg];
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    r[i] = st[size_t(i) * P];
    s[i] = st[size_t(kReg + i) * P];
  }
  // Unless every lane has the same length (one plain store of the whole group
  // at the end), the end points OR their lanes' words in: clear those lanes.
  if (!same_end(lt, lanes, C)) {
#pragma unroll 1
    for (int i = 0; i < 2 * kReg; ++i) atomicAnd(st + size_t(i) * P, ~alive);
  }
  uint32_t *zb0 = zs + threadIdx.x, *zb1 = zs + 32 * kRaggedThreads + threadIdx.x;
  KgFeed fd = kg_feed<false>(r, s, 0u);
  const uint32_t NT = uint32_t((C + 31) >> 5);      // lengths are at most 2^34
#pragma unroll 1
  for (uint32_t T = 0; T < NT; ++T) {
    const uint64_t t0 = uint64_t(T) << 5;
    uint32_t *cur = (T & 1) ? zb1 : zb0, *prev = (T & 1) ? zb0 : zb1;
    const uint32_t ends = tile_ends(lt, lanes, t0);
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
      cur[c * kRaggedThreads] = lop3<kXorAnd>(r[0], s[0], alive);  // (r0 ^ s0) & alive
      clock_kg_from<false>(r, s, fd, 0u);
      fd = kg_feed<false>(r, s, 0u);         // the next clock's, inside this iteration
      if ((ends >> c) & 1u) {                  // some lanes have run their length
        const uint32_t m = lanes_ending(lt, lanes, t0 + c + 1);
        snapshot(st, P, r, s, m, pad);
        alive &= ~m;
      }
      if ((c & 3) == 3 && T > 0)
        ragged_slice<LAYOUT>(prev, lt, grow, lanes, t0 - 32, 32, C, c >> 2);
    }
  }
  // the last tile (possibly partial)
  const uint64_t tl = uint64_t(NT - 1) << 5;
  ragged_tile<LAYOUT>(((NT - 1) & 1) ? zb1 : zb0, lt, grow, lanes, tl,
                      C - tl >= 32 ? 32 : int(C - tl), C);
}

template <int LAYOUT>
cudaError_t launch_ragged_layout(const RaggedArgs &a, cudaStream_t st) {
  const cudaError_t e = cudaFuncSetAttribute(
      ragged_kernel<LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kRaggedSmem));
  if (e != cudaSuccess) return e;
  const uint32_t blocks = (a.G + kRaggedThreads - 1) / kRaggedThreads;
  ragged_kernel<LAYOUT><<<blocks, kRaggedThreads, kRaggedSmem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ragged(const RaggedArgs &a, int layout, cudaStream_t st) {
  switch (layout) {
    case MICKEY_LAYOUT_BITSLICED_U32: return launch_ragged_layout<MICKEY_LAYOUT_BITSLICED_U32>(a, st);
    case MICKEY_LAYOUT_BYTES: return launch_ragged_layout<MICKEY_LAYOUT_BYTES>(a, st);
    case MICKEY_LAYOUT_U32: return launch_ragged_layout<MICKEY_LAYOUT_U32>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mickey
