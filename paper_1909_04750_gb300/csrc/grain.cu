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
//          as H0 + b63 H1, H0 and H1 of LFSR bits only             10 ops
//   init   z is added into both new bits (into the LFSR's last XOR)  +1
// Keystream words go to a ring of 160 words per thread in shared memory
// (two bodies of 80 clocks fill five 32-clock tiles); after each body the
// finished tiles are emitted: as they are (bitsliced layout) or, for
// row-major bytes, transposed by the two-pass in-place block swaps also used
// for MICKEY, on the tile's rows in reverse order, since Grain's bytes hold
// the first keystream bit in the least significant bit.  The bytes layout
// stages eight tiles of every row so that each row goes out as whole
// 32-byte sectors; the staging (1 KiB per thread) lives in tensor memory,
// not shared memory, so that the shared memory of an SM (the rings) holds
// two warps per SM sub-partition.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/grain.h"
#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "grain_clock.cuh"
#include "internal.h"

namespace mickey {
namespace {

using namespace grainc;

struct GrainArgs {
  uint32_t *state;      // 160 x Gpad words: s0..s79 then b0..b79
  uint32_t G, Gpad;
  uint64_t n;
  uint64_t n_bits;
  void *out;
  uint32_t last_mask;   // valid lanes of the last group
};

// Clocks per queue item: a multiple of the ring (160) and of the row staging
// (8 tiles = 256 clocks), so that every item starts on a fresh body, tile and
// staged block.
constexpr uint64_t kChunk = 1280;

struct GrainQueue {
  uint32_t *counter;    // items taken, zero at launch
  uint32_t *flags;      // per warp-group: chunks finished, zero at launch
  uint32_t W;           // warp-groups
  uint64_t chunk;       // clocks per item
  uint64_t n_chunks;
  uint32_t spin_limit;  // polls of ~256 ns before a wait gives up
  int *err;
};

// Row staging of the bytes layout: the transposed words of 8 consecutive
// tiles per lane, so that each row goes out as one whole 32-byte sector (two
// 16-byte stores) instead of 4-byte pieces.
constexpr int kStage = 8;

// Blocks of the bytes layout: eight warps, two per lane quarter of tensor
// memory (warp w: lanes 32 (w % 4) .. + 31, columns 256 (w / 4) .. + 255).
// A kernel that allocates tensor memory runs one block per SM (that is what
// the occupancy calculator answers for it, whatever its other resources),
// so the block takes all 512 columns of the SM; its rings fill 160 KiB of
// shared memory and its 256 threads the register file.
constexpr int kGrainBytesThreads = 256;
constexpr uint32_t kTmemCols = 512;

template <int LAYOUT>
__host__ __device__ constexpr int grain_threads() {
  return LAYOUT == MICKEY_LAYOUT_BYTES ? kGrainBytesThreads : kGrainThreads;
}

// Tensor memory (TMEM) used as plain storage: a block allocates columns, a
// warp reads and writes 32-bit words of its own 32 lanes (lane = the
// thread's lane, lanes 32 (warp % 4) .. + 31) with warp-wide instructions.
// Address: lane in bits 31..16, column in bits 15..0.
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2,
                                         uint32_t v3) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};"
               :: "r"(taddr), "r"(v0), "r"(v1), "r"(v2), "r"(v3) : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
// Columns taddr .. taddr + 15 of the thread's lane; returns once they are in
// registers (the load and its wait in one statement, so that no use of the
// registers can be scheduled before the wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&w)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
        "=r"(w[7]), "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]),
        "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
      : "r"(taddr)
      : "memory");
}

// Bytes layout: warp 0 allocates the block's columns (the address goes
// through shared memory to every warp); returns the warp's base address
// (its lane quarter and its 256 columns).  Other layouts use no tensor memory.
template <int LAYOUT>
__device__ __forceinline__ uint32_t tmem_open(uint32_t *slot) {
  if constexpr (LAYOUT == MICKEY_LAYOUT_BYTES) {
    if (threadIdx.x < 32) {
      const uint32_t dst = uint32_t(__cvta_generic_to_shared(slot));
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                   :: "r"(dst), "r"(kTmemCols) : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t warp = threadIdx.x >> 5;
    return *slot + (((warp & 3u) * 32u) << 16) + (warp >> 2) * 256u;
  } else {
    return 0;
  }
}

// Every warp's tensor-memory accesses have completed; warp 0 frees the columns.
template <int LAYOUT>
__device__ __forceinline__ void tmem_close(const uint32_t *slot) {
  if constexpr (LAYOUT == MICKEY_LAYOUT_BYTES) {
    __syncwarp();
    tmem_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                   :: "r"(*slot), "r"(kTmemCols) : "memory");
  }
}

// Emit the 32-clock tile k of the call (clocks 32k .. 32k+nb-1) held in zb
// (word c = clock 32k + c, bit l = lane l; stride kRingStride) of group g.
// Bitsliced: stored as it is.  Bytes: transposed and staged in tensor memory
// at tm (the warp's lanes, 256 columns: column 32r + 4 slot + q holds the
// word of lane 31 - r - 8q for the tile in staging slot k % 8); the staged
// tiles are written out after the last tile of each aligned block of 8 and
// after the call's last tile.  The bytes path runs warp-wide instructions:
// every lane of the warp takes it, lanes outside `mask` store nothing.
template <int LAYOUT>
__device__ __forceinline__ void grain_emit(uint32_t *zb, uint32_t tm, const GrainArgs &a,
                                           uint32_t g, uint64_t k, int nb, uint32_t mask) {
  constexpr int S = kRingStride;
  const uint64_t t0 = k << 5;
  if constexpr (LAYOUT == MICKEY_LAYOUT_BITSLICED_U32) {
    if (mask == 0) return;                 // a lane past the last group: nothing to store
    uint32_t *o = static_cast<uint32_t *>(a.out) + size_t(g) * a.n_bits + t0;
    if (nb == 32 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint4 v;
        v.x = zb[(4 * j + 0) * S] & mask;
        v.y = zb[(4 * j + 1) * S] & mask;
        v.z = zb[(4 * j + 2) * S] & mask;
        v.w = zb[(4 * j + 3) * S] & mask;
        reinterpret_cast<uint4 *>(o)[j] = v;
      }
    } else {
      for (int c = 0; c < nb; ++c) o[c] = zb[c * S] & mask;
    }
  } else {
    // The tile is transposed with its rows taken in reverse order (row i =
    // clock 31 - i): the transposed row of lane l then holds clock c in bit
    // c, the order of Grain's bytes (first keystream bit in the least
    // significant bit), with no bit reversal.
    // pass 1: block swaps of size 4, 2, 1 within each 8 rows
#pragma unroll 1
    for (int j = 0; j < 4; ++j) {
      uint32_t v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = zb[(31 - 8 * j - q) * S];
      swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
      swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
      swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
      swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
      swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
      swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
      for (int q = 0; q < 8; ++q) zb[(31 - 8 * j - q) * S] = v[q];
    }
    // pass 2: block swaps of size 16 and 8; row r + 8q is lane 31 - r - 8q
    const int slot = int(k & (kStage - 1));
    __syncwarp();
#pragma unroll 1
    for (int r = 0; r < 8; ++r) {
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = zb[(31 - r - 8 * q) * S];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes<false>(v[0], v[1]);
      swap_bytes<false>(v[2], v[3]);
      tmem_st4(tm + uint32_t(32 * r + 4 * slot), v[0], v[1], v[2], v[3]);
    }
    const bool last = t0 + uint64_t(nb) >= a.n_bits;
    if (slot == kStage - 1 || last) {
      // write tiles k - slot .. k of every valid lane
      tmem_wait_st();
      const uint32_t pitch = uint32_t((a.n_bits + 7) >> 3);
      const uint64_t kA = k - uint64_t(slot);
      uint8_t *base = static_cast<uint8_t *>(a.out) + 32ull * g * pitch + kA * 4;
      const bool sector = slot == kStage - 1 && nb == 32 && (pitch & 15u) == 0 &&
                          (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
      // bytes of the staged block that belong to the call
      const uint64_t bytes = ((kA << 5) + ((uint64_t(slot) << 5) + uint64_t(nb)) + 7) / 8 -
                             ((kA << 5) >> 3);
#pragma unroll 1
      for (int r = 0; r < 8; ++r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {            // slots 4h .. 4h + 3: bytes 16h .. 16h + 15
          uint32_t w[16];                        // w[4 j + q]: slot 4h + j of lane 31 - r - 8q
          __syncwarp();
          tmem_ld16(tm + uint32_t(32 * r + 16 * h), w);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int l = 31 - r - 8 * q;
            if (!((mask >> l) & 1u)) continue;
            uint8_t *o = base + uint64_t(uint32_t(l) * pitch) + 16 * h;
            if (sector) {
              *reinterpret_cast<uint4 *>(o) = make_uint4(w[q], w[4 + q], w[8 + q], w[12 + q]);
            } else {
#pragma unroll
              for (int by = 0; by < 16; ++by)
                if (uint64_t(16 * h + by) < bytes)
                  o[by] = uint8_t(w[4 * (by >> 2) + q] >> (8 * (by & 3)));
            }
          }
        }
      }
    }
  }
}

// Clocks [t_a, t_b) of the call for group g (t_a a multiple of kChunk, so
// that its bodies, ring slots, tiles and staged blocks line up), from and back
// to the state in HBM; `live` is false for the lanes of a warp past the last
// group, which clock a copy of group 0's state and store nothing.
template <int LAYOUT>
__device__ __forceinline__ void grain_piece(const GrainArgs &a, uint32_t g, bool live,
                                            uint64_t t_a, uint64_t t_b, uint32_t *zb,
                                            uint32_t tm) {
  const size_t P = a.Gpad;
  const uint32_t gs = live ? g : 0;
  uint32_t s[kG], b[kG];
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    s[i] = a.state[size_t(i) * P + gs];
    b[i] = a.state[size_t(kG + i) * P + gs];
  }
  const uint32_t mask = !live ? 0u : g == a.G - 1 ? a.last_mask : ~0u;
  const uint64_t n = t_b - t_a;
  const uint64_t full = n / kG;             // whole bodies of 80 clocks
  uint64_t emitted = 0;                     // tiles of this piece emitted so far
#pragma unroll 1
  for (uint64_t j = 0; j < full; ++j) {
    grain_body<false>(s, b, zb + (j & 1) * kG * kRingStride);
    const uint64_t done = (j + 1) * kG;
#pragma unroll 1
    for (; (emitted + 1) * 32 <= done; ++emitted)
      grain_emit<LAYOUT>(zb + ((emitted * 32) % kRing) * kRingStride, tm, a, g,
                         (t_a >> 5) + emitted, 32, mask);
  }
  const int rem = int(n - full * kG);
  if (rem) {
    uint32_t *zt = zb + (full & 1) * kG * kRingStride;
#pragma unroll 1
    for (int c = 0; c < rem; ++c) zt[c * kRingStride] = grain_clock_shift(s, b);
  }
#pragma unroll 1
  for (; emitted * 32 < n; ++emitted) {
    const int nb = int(min(uint64_t(32), n - emitted * 32));
    uint32_t *zt = zb + ((emitted * 32) % kRing) * kRingStride;
    for (int c = nb; c < 32; ++c) zt[c * kRingStride] = 0u;   // past the call's last clock
    grain_emit<LAYOUT>(zt, tm, a, g, (t_a >> 5) + emitted, nb, mask);
  }
  if (live) {
#pragma unroll
    for (int i = 0; i < kG; ++i) {
      a.state[size_t(i) * P + g] = s[i];
      a.state[size_t(kG + i) * P + g] = b[i];
    }
  }
}

__device__ __forceinline__ uint32_t grain_load_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void grain_store_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Persistent launch (every block resident; used when there are more
// warp-groups than resident warps): warps take items from a queue,
// item i = chunk i / W of warp-group i % W (W warp-groups of 32 groups,
// chunks of kChunk clocks), so that all first chunks come first.  Chunk k of
// a warp-group starts from the state its chunk k - 1 published: the warp
// waits (bounded) until the warp-group's flag reaches k.  That item was taken
// from the queue earlier by a warp that is running, so the wait ends; if it
// runs out the error flag is raised and the item is skipped (the call's
// output and state are then undefined, and grain_sync reports it).  Every SM
// sub-partition keeps its full share of warps until the queue runs dry.
template <int LAYOUT>
__global__ void __launch_bounds__(grain_threads<LAYOUT>())
    grain_keystream_kernel(GrainArgs a, GrainQueue q) {
  // shared memory: each warp's keystream ring (kRing words per thread,
  // [word][lane]); the bytes layout's row staging is in tensor memory
  extern __shared__ __align__(16) uint32_t ring[];
  __shared__ uint32_t tmem_slot;
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t *zb = ring + (threadIdx.x >> 5) * (kRing * kRingStride) + lane;
  const uint32_t tm = tmem_open<LAYOUT>(&tmem_slot);
  const uint64_t items = uint64_t(q.W) * q.n_chunks;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(q.counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= items) break;
    const uint32_t k = item / q.W, w = item % q.W;
    if (k > 0) {   // every lane acquires the predecessor's published state
      uint32_t it = 0;
      bool ok = true;
      while (grain_load_acquire(q.flags + w) < k) {
        if (++it > q.spin_limit) {
          ok = false;
          break;
        }
        __nanosleep(256);
      }
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicOr(q.err, kErrTimeout);
        continue;
      }
    }
    const uint32_t g = w * 32 + lane;
    const uint64_t t_a = uint64_t(k) * q.chunk;
    const uint64_t t_b = min(a.n_bits, t_a + q.chunk);
    grain_piece<LAYOUT>(a, g, g < a.G, t_a, t_b, zb, tm);
    __threadfence();
    __syncwarp();
    if (lane == 0) grain_store_release(q.flags + w, k + 1);
  }
  tmem_close<LAYOUT>(&tmem_slot);
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

// Copy `bytes` bytes of src into rows of row_bytes bytes, stride_words apart:
// 4-byte cp.async copies (all in flight at once; the caller waits) when src
// is 4-byte aligned, byte loads otherwise and for a last partial word.
__device__ __forceinline__ void stage(const uint8_t *src, uint64_t bytes, uint32_t *dst,
                                      int row_bytes, int stride_words) {
  const int row_words = row_bytes / 4;
  const bool aligned = (reinterpret_cast<uintptr_t>(src) & 3u) == 0;
  for (uint64_t w = threadIdx.x; w * 4 < bytes; w += kInitT) {
    uint32_t *d = dst + (w / row_words) * stride_words + w % row_words;
    if (aligned && w * 4 + 4 <= bytes) {
      const uint32_t da = uint32_t(__cvta_generic_to_shared(d));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(da),
                   "l"(reinterpret_cast<const uint32_t *>(src) + w) : "memory");
    } else {
      uint32_t v = 0;
      for (int k = 0; k < 4 && w * 4 + k < bytes; ++k) v |= uint32_t(src[w * 4 + k]) << (8 * k);
      *d = v;
    }
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
  asm volatile("cp.async.wait_all;" ::: "memory");
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
  // 160 clocks with z fed back: one 80-clock rotation, run twice (the
  // mapping of slots to register bits is back at the start after 80)
#pragma unroll 1
  for (int rep = 0; rep < 2; ++rep) grain_body<true>(s, b, nullptr);
  const size_t P = a.Gpad;
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    a.state[size_t(i) * P + g] = s[i];
    a.state[size_t(kG + i) * P + g] = b[i];
  }
}

// One thread per group for the whole call (used when every warp-group fits
// in the resident warps at once, so that the queue would add waits and no
// parallelism: a warp-group's chunks cannot overlap).
template <int LAYOUT>
__global__ void __launch_bounds__(grain_threads<LAYOUT>()) grain_grid_kernel(GrainArgs a) {
  extern __shared__ __align__(16) uint32_t ring[];
  __shared__ uint32_t tmem_slot;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t tm = tmem_open<LAYOUT>(&tmem_slot);
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g - lane < a.G)   // the warp holds a group; its lanes past the last group store nothing
    grain_piece<LAYOUT>(a, g, g < a.G, 0, a.n_bits,
                        ring + (threadIdx.x >> 5) * (kRing * kRingStride) + lane, tm);
  tmem_close<LAYOUT>(&tmem_slot);
}

template <int LAYOUT>
cudaError_t launch_grain_layout(const GrainArgs &a, const GrainQueue &q, int sm_count,
                                int force, cudaStream_t st) {
  constexpr int T = grain_threads<LAYOUT>();
  const size_t smem = size_t(kRing) * T * 4;
  cudaError_t e = cudaFuncSetAttribute(grain_keystream_kernel<LAYOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(grain_grid_kernel<LAYOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem));
  if (e != cudaSuccess) return e;
  // the rings of two blocks need the largest shared-memory carveout
  e = cudaFuncSetAttribute(grain_keystream_kernel<LAYOUT>,
                           cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(grain_grid_kernel<LAYOUT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           int(cudaSharedmemCarveoutMaxShared));
  if (e != cudaSuccess) return e;
  int per_sm = 0, per_sm_grid = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grain_keystream_kernel<LAYOUT>, T,
                                                    smem);
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_grid, grain_grid_kernel<LAYOUT>, T,
                                                    smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || per_sm_grid < 1) return cudaErrorInvalidConfiguration;
  // the blocks resident on an SM must never ask for more tensor memory than it
  // has (an allocation that cannot be met waits)
  if (LAYOUT == MICKEY_LAYOUT_BYTES &&
      uint32_t(std::max(per_sm, per_sm_grid)) * kTmemCols > 512u)
    return cudaErrorInvalidConfiguration;
  // The grid launch when every warp-group gets a warp of its own, even if
  // some SMs then get no block: a warp-group's clocks are one sequential
  // chain, so spreading chunks over more warps (the queue) only adds waits
  // (2^20 bytes-layout instances: 6.9 Tbit/s on 128 SMs against 5.7 through
  // the queue on all 152).  `force` = 1: always the queue.
  const uint64_t slots = uint64_t(per_sm) * sm_count * (T / 32);
  if (q.W <= slots && force != 1) {
    grain_grid_kernel<LAYOUT><<<(a.G + T - 1) / T, T, smem, st>>>(a);
    return cudaGetLastError();
  }
  // every block resident (the waits need it); no more warps than items
  const uint64_t items = uint64_t(q.W) * q.n_chunks;
  const uint64_t want = (items + T / 32 - 1) / (T / 32);
  const uint32_t blocks = uint32_t(std::min<uint64_t>(uint64_t(per_sm) * sm_count, want));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(T);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, grain_keystream_kernel<LAYOUT>, a, q);
}

// Logic ops per clock per 32-lane group, as written above (keystream clock
// including z, or an initialisation clock).
constexpr int kGrainOps = 10 + 3 + 23;
constexpr int kGrainInitOps = kGrainOps + 1;

}  // namespace
}  // namespace mickey

using namespace mickey;

struct grain_streams {
  size_t n = 0;
  uint32_t G = 0, Gpad = 0;
  uint32_t *d_state = nullptr;
  uint8_t *d_inputs = nullptr;   // host inputs staged: keys (10n), ivs (8n)
  uint32_t *d_queue = nullptr;   // item counter, then one flag per warp-group
  int *d_err = nullptr;
  cudaStream_t stream = nullptr;
  uint64_t pos = 0;
  int sm_count = 0;
  uint32_t spin_limit = 1u << 24;
  int force = -1;                // MICKEY_GRAIN_QUEUE=1: always the queue-fed launch,
                                 // =0 (the default): the grid launch when every warp-group fits
};

namespace {

int grain_fail(int code, const char *msg) { return set_error(code, msg); }

void grain_release(grain_streams *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->d_state);
  cudaFree(s->d_inputs);
  cudaFree(s->d_queue);
  cudaFree(s->d_err);
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
  int dev = 0;
  bool ok = cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) ==
                cudaSuccess &&
            cudaMalloc(&s->d_state, size_t(2 * kG) * s->Gpad * 4) == cudaSuccess &&
            cudaMalloc(&s->d_queue, (1 + size_t(s->Gpad / 32)) * 4) == cudaSuccess &&
            cudaMalloc(&s->d_err, sizeof(int)) == cudaSuccess &&
            cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream) == cudaSuccess;
  if (const char *v = getenv("MICKEY_SPIN_LIMIT")) {
    const long long l = atoll(v);
    if (l > 0 && l < (1ll << 31)) s->spin_limit = uint32_t(l);
  }
  if (const char *v = getenv("MICKEY_GRAIN_QUEUE")) s->force = atoi(v) != 0 ? 1 : 0;
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
  const uint32_t W = (s->G + 31) / 32;
  GrainQueue q{s->d_queue, s->d_queue + 1, W, kChunk, (n_bits + kChunk - 1) / kChunk,
               s->spin_limit, s->d_err};
  if (cudaMemsetAsync(s->d_queue, 0, (1 + size_t(W)) * 4, s->stream) != cudaSuccess)
    return grain_fail(MICKEY_E_CUDA, "queue reset");
  const cudaError_t e =
      layout == MICKEY_LAYOUT_BYTES
          ? launch_grain_layout<MICKEY_LAYOUT_BYTES>(a, q, s->sm_count, s->force, s->stream)
          : launch_grain_layout<MICKEY_LAYOUT_BITSLICED_U32>(a, q, s->sm_count, s->force,
                                                             s->stream);
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
  int flag = 0;
  if (cudaMemcpy(&flag, s->d_err, sizeof flag, cudaMemcpyDeviceToHost) != cudaSuccess)
    return grain_fail(MICKEY_E_CUDA, "error flag copy");
  if (flag) {
    cudaMemset(s->d_err, 0, sizeof(int));
    return grain_fail(MICKEY_E_TIMEOUT, "a device-side wait timed out");
  }
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
