// Batched generation: many streams of uneven keystream length and IV
// length in one persistent launch.
//
// Plan (host, once per shape): streams are sorted by keystream length,
// longest first, and packed 32 at a time into bitsliced groups, so the
// lanes of a group need similar numbers of clocks; a group runs as many
// clocks as its longest lane and each lane keeps only its own bits.  Each
// stream's output is its own row-major byte string at a 16-byte aligned
// offset (in the caller's stream order).
//
// Run (device, captured once as a CUDA graph and replayed): key/IV loading
// through the sorting permutation, preclock, then the keystream.  The first
// n_split groups, the longest, run one per warp (split path: the warp clocks
// one group, several times less time per clock, for the groups that bound
// the run); the rest 32 consecutive groups per warp item, one per thread.
// Items are taken from atomic counters longest first (longest processing
// time first).  Two arrangements (the split mode):
//   shared  one persistent kernel: its warps take the split items first,
//           then the thread items.  A long split warp keeps its SM
//           sub-partition to itself, which is best for one batch's critical
//           path.
//   own     the split groups in a kernel of one-warp blocks (one per SM
//           sub-partition) beside the thread kernel, as parallel branches of
//           the graph.  A block of short thread items then retires, and frees
//           its registers for the next batch's work, however long the split
//           warps run: the arrangement for batches back to back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "internal.h"
#include "split.cuh"

using namespace mickey;

namespace {

constexpr int kBatchThreads = 128;

struct BatchParams {  // device-side, written before each graph launch
  uint8_t *out;
};

struct BatchArgs {
  const uint32_t *state;     // kStateRows x Gpad, group order
  uint32_t G, Gpad;
  const uint64_t *slot_off;  // 32*Gpad: byte offset of the slot's stream in out
  const uint64_t *slot_bits; // 32*Gpad: keystream bits of the slot's stream (0: padding)
  const uint64_t *group_bits;// Gpad: clocks of the group (its longest lane)
  uint32_t n_split;          // groups 0..n_split-1 run on a whole warp each
  uint32_t split_items;      // split items this kernel takes (n_split, or 0 in "own" mode)
  uint32_t n_items;          // split_items + ceil((G - n_split) / 32)
  uint32_t *queue;           // [0]: split-group counter, [1]: item counter, zero at launch
  const BatchParams *params;
};

// Store word w (memory byte order) of the lane's tile t, clipped to the
// lane's n_bits (bits past the end of a last partial byte are zeroed).
__device__ __forceinline__ void store_ragged(uint8_t *out, const BatchArgs &a, uint64_t slot,
                                             uint32_t t, uint32_t w) {
  const uint64_t bits = __ldg(a.slot_bits + slot);
  const uint64_t b0 = uint64_t(t) << 5;
  if (b0 >= bits) return;
  uint8_t *o = out + __ldg(a.slot_off + slot) + (b0 >> 3);
  const uint64_t left = bits - b0;
  if (left >= 32) {
    *reinterpret_cast<uint32_t *>(o) = w;
    return;
  }
  const uint32_t keep_be = ~0u << (32 - uint32_t(left));            // big-endian bit order
  w &= __byte_perm(keep_be, 0u, 0x0123);                               // to memory order
  const int nbytes = int((left + 7) >> 3);
  for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(w >> (8 * b));
}

// One eighth of the emission of tile t (see the keystream kernels: slices
// 0-3 swap blocks of size 4, 2, 1 in place, slices 4-7 swap blocks of size
// 16, 8 and store), for ragged rows.
__device__ __forceinline__ void batch_slice(uint32_t *z, uint8_t *out, const BatchArgs &a,
                                            uint32_t g, uint32_t t, int j) {
  if (j < 4) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = z[(8 * j + k) * kBatchThreads];
    swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
    swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
    swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
    swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
    swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
    swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) z[(8 * j + k) * kBatchThreads] = v[k];
  } else {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * (j - 4) + h;
      uint32_t v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = z[(k + 8 * q) * kBatchThreads];
      swap_halves(v[0], v[2]);
      swap_halves(v[1], v[3]);
      swap_bytes<true>(v[0], v[1]);
      swap_bytes<true>(v[2], v[3]);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        store_ragged(out, a, uint64_t(g) * 32 + (31 - k - 8 * q), t, v[q]);
    }
  }
}

template <int U>
__device__ __forceinline__ void batch_group(const BatchArgs &a, uint8_t *out, uint32_t g,
                                            uint32_t *zb0, uint32_t *zb1) {
  const size_t P = a.Gpad;
  uint32_t r[kReg], s[kReg];
  const uint32_t *src = a.state + g;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    r[i] = src[size_t(i) * P];
    s[i] = src[size_t(kReg + i) * P];
  }
  const uint64_t clocks = a.group_bits[g];
  const uint32_t full = uint32_t(clocks >> 5);
#pragma unroll 1
  for (uint32_t tile = 0; tile < full; ++tile) {
    uint32_t *cur = (tile & 1) ? zb1 : zb0;
    uint32_t *prev = (tile & 1) ? zb0 : zb1;
#pragma unroll 1
    for (int c = 0; c < 32; c += U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cur[(c + u) * kBatchThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      }
      if (tile > 0 && (c & 3) == 0) batch_slice(prev, out, a, g, tile - 1, c >> 2);
    }
  }
  if (full > 0) {
#pragma unroll 1
    for (int j = 0; j < 8; ++j) batch_slice((full & 1) ? zb0 : zb1, out, a, g, full - 1, j);
  }
  const int rem = int(clocks & 31);
  if (rem) {
    uint32_t *cur = (full & 1) ? zb1 : zb0;
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
      if (c < rem) {
        cur[c * kBatchThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      } else {
        cur[c * kBatchThreads] = 0u;
      }
    }
#pragma unroll 1
    for (int j = 0; j < 8; ++j) batch_slice(cur, out, a, g, full, j);
  }
}

// Store word w (memory byte order) of tile t of a row at o with `bits`
// keystream bits (split path: row address and length held in registers).
__device__ __forceinline__ void store_row(uint8_t *o, uint64_t bits, uint32_t t, uint32_t w) {
  const uint64_t b0 = uint64_t(t) << 5;
  if (b0 >= bits) return;
  o += b0 >> 3;
  const uint64_t left = bits - b0;
  if (left >= 32) {
    *reinterpret_cast<uint32_t *>(o) = w;
    return;
  }
  w &= __byte_perm(~0u << (32 - uint32_t(left)), 0u, 0x0123);
  const int nbytes = int((left + 7) >> 3);
  for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(w >> (8 * b));
}

// One warp per group (split path).  Not inlined: as a function of its own it
// gets a register allocation of its own (about 120 registers, no spills)
// instead of sharing the one-thread-per-group path's 255, which made its
// clock about 20 % slower.  The tile's bits come back transposed
// (clock c in bit c of lane l's word), reversed so that the tile's first
// clock comes first, and put in memory byte order.
__device__ __noinline__ void split_group(const uint32_t *state, size_t P, uint32_t g,
                                            uint64_t clocks, uint8_t *row, uint64_t bits,
                                            uint32_t lane, uint32_t *zbuf0, uint32_t *zbuf1) {
  SplitLane k;
  split_lane_init(lane, k);
  uint32_t r[4], s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = int(4 * lane) + q;
    r[q] = i < kReg ? state[size_t(i) * P + g] : 0u;
    const int is = split_s_bit(int(lane), q);
    s[q] = is >= 0 && is < kReg ? state[size_t(kReg + is) * P + g] : 0u;
  }
  const uint32_t full = uint32_t(clocks >> 5);
#pragma unroll 1
  for (uint32_t t = 0; t < full; ++t) {
    const uint32_t mine = split_tile<kSplitUnroll>(r, s, k, lane, zbuf0, zbuf1, 32);
    store_row(row, bits, t, __byte_perm(__brev(mine), 0u, 0x0123));
  }
  const int rem = int(clocks & 31);
  if (rem) {
    const uint32_t mine = split_tile<kSplitUnroll>(r, s, k, lane, zbuf0, zbuf1, rem);
    store_row(row, bits, full, __byte_perm(__brev(mine), 0u, 0x0123));
  }
  __syncwarp();
}

// Split kernel: one-warp blocks take the split groups (0 .. n_split-1,
// longest first) one at a time.
__global__ void __launch_bounds__(32) batch_split_kernel(BatchArgs a) {
  __shared__ uint32_t zs[64];
  const uint32_t lane = threadIdx.x;
  uint8_t *out = a.params->out;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_split) break;
    const uint64_t slot = uint64_t(item) * 32 + lane;
    split_group(a.state, a.Gpad, item, a.group_bits[item], out + a.slot_off[slot],
                a.slot_bits[slot], lane, zs, zs + 32);
  }
}

// Persistent kernel: its first split_items items are split groups, run by
// a whole warp each; then items of 32 consecutive groups from group n_split
// on, one group per thread.
template <int U>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(BatchArgs a) {
  __shared__ uint32_t zs[2 * 32 * kBatchThreads];
  const uint32_t lane = threadIdx.x & 31u;
  uint8_t *out = a.params->out;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.queue + 1, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    if (item < a.split_items) {
      // the warp's own 32 columns of rows 0 and 1 of the tile buffer
      const uint64_t slot = uint64_t(item) * 32 + lane;
      uint32_t *zb = zs + (threadIdx.x & ~31u);
      split_group(a.state, a.Gpad, item, a.group_bits[item], out + a.slot_off[slot],
                  a.slot_bits[slot], lane, zb, zb + kBatchThreads);
      continue;
    }
    const uint32_t g = a.n_split + (item - a.split_items) * 32 + lane;
    if (g < a.G)
      batch_group<U>(a, out, g, zs + threadIdx.x, zs + 32 * kBatchThreads + threadIdx.x);
  }
}

bool valid_unroll(int u) { return u == 2 || u == 4; }

}  // namespace

struct mickey_batch {
  size_t n = 0;
  uint32_t G = 0, Gpad = 0;
  uint64_t out_bytes = 0, max_clocks = 0, total_clocks = 0;
  std::vector<uint64_t> offsets;  // per stream, caller order
  std::vector<uint64_t> group_clocks;  // longest first
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  int unroll = 4, blocks_per_sm = 2;
  uint64_t split_clocks = 0;      // groups longer than this use the split path (0: none)
  uint32_t n_split = 0;
  int split_mode = MICKEY_BATCH_SPLIT_SHARED;
  // device
  uint8_t *d_in = nullptr;        // keys (10n), ivs (10n), iv_lens (4n) in caller order
  uint32_t *d_perm = nullptr;     // 32*Gpad
  uint64_t *d_slot = nullptr;     // slot_off (32*Gpad), slot_bits (32*Gpad), group_bits (Gpad)
  uint32_t *d_state = nullptr, *d_scratch = nullptr, *d_queue = nullptr;
  int *d_err = nullptr;
  BatchParams *d_params = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void batch_release(mickey_batch *b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_in);
  cudaFree(b->d_perm);
  cudaFree(b->d_slot);
  cudaFree(b->d_state);
  cudaFree(b->d_scratch);
  cudaFree(b->d_queue);
  cudaFree(b->d_err);
  cudaFree(b->d_params);
  delete b;
}

// Capture load + preclock, then the split kernel and the thread kernel as
// two parallel branches, into a graph.
cudaError_t capture(mickey_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  cudaStream_t cs = nullptr, cs2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const size_t n = b->n;
    cudaMemsetAsync(b->d_queue, 0, 2 * sizeof(uint32_t), cs);
    LoadArgs la{b->d_in, b->d_in + 10 * n, reinterpret_cast<const uint32_t *>(b->d_in + 20 * n),
                n, b->d_perm, b->G, b->Gpad, b->d_scratch, b->d_err};
    launch_init(la, b->d_state, cs);
    const bool own = b->split_mode == MICKEY_BATCH_SPLIT_OWN && b->n_split;
    const uint32_t split_items = own ? 0u : b->n_split;
    BatchArgs ba{b->d_state, b->G, b->Gpad, b->d_slot, b->d_slot + 32 * size_t(b->Gpad),
                 b->d_slot + 64 * size_t(b->Gpad), b->n_split, split_items,
                 split_items + (b->G - b->n_split + 31) / 32, b->d_queue, b->d_params};
    if (own) {   // the split groups on a branch of their own
      cudaEventRecord(fork, cs);
      cudaStreamWaitEvent(cs2, fork, 0);
      const uint32_t warps = std::min<uint32_t>(b->n_split, uint32_t(b->sm_count) * 4u);
      batch_split_kernel<<<warps, 32, 0, cs2>>>(ba);
      cudaEventRecord(join, cs2);
    }
    if (ba.n_items) {
      const uint32_t grid = uint32_t(b->sm_count * b->blocks_per_sm);
      if (b->unroll == 2)
        batch_kernel<2><<<grid, kBatchThreads, 0, cs>>>(ba);
      else
        batch_kernel<4><<<grid, kBatchThreads, 0, cs>>>(ba);
    }
    if (own) cudaStreamWaitEvent(cs, join, 0);
    e = cudaStreamEndCapture(cs, &b->graph);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (fork) cudaEventDestroy(fork);
  if (join) cudaEventDestroy(join);
  if (cs2) cudaStreamDestroy(cs2);
  if (cs) cudaStreamDestroy(cs);
  return e;
}

int copy_inputs(mickey_batch *b, const void *keys, const void *ivs, int mem) {
  const cudaMemcpyKind kind =
      mem == MICKEY_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (cudaMemcpyAsync(b->d_in, keys, 10 * b->n, kind, b->stream) != cudaSuccess ||
      cudaMemcpyAsync(b->d_in + 10 * b->n, ivs, 10 * b->n, kind, b->stream) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "key/IV upload");
  return MICKEY_OK;
}

}  // namespace

extern "C" {

MICKEY_API mickey_batch *mickey_batch_create(const uint32_t *iv_lens, const uint64_t *n_bits,
                                             size_t n, void *cuda_stream) {
  if (!n_bits || n == 0 || n > (size_t(1) << 31)) {
    set_error(MICKEY_E_ARG, "n_bits must not be NULL and 0 < n <= 2^31");
    return nullptr;
  }
  for (size_t i = 0; i < n; ++i) {
    if (n_bits[i] > MICKEY_MAX_STREAM_BITS) {
      set_error(MICKEY_E_LIMIT, "a stream asks for more than 2^40 keystream bits");
      return nullptr;
    }
    if (iv_lens && iv_lens[i] > MICKEY_MAX_IV_BITS) {
      set_error(MICKEY_E_IVLEN, "an IV length exceeds 80 bits");
      return nullptr;
    }
  }
  mickey_batch *b = new (std::nothrow) mickey_batch;
  if (!b) {
    set_error(MICKEY_E_OOM, "host allocation failed");
    return nullptr;
  }
  b->n = n;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->G = uint32_t((n + 31) / 32);
  b->Gpad = (b->G + 31u) & ~31u;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);

  // longest first; ties keep the caller's order
  std::vector<uint32_t> order(n);
  std::iota(order.begin(), order.end(), 0u);
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return n_bits[x] > n_bits[y]; });
  b->offsets.resize(n);
  uint64_t off = 0;
  for (size_t i = 0; i < n; ++i) {  // caller order, 16-byte aligned rows
    b->offsets[i] = off;
    off += ((n_bits[i] + 7) / 8 + 15) & ~uint64_t(15);
  }
  b->out_bytes = off;
  b->group_clocks.resize(b->G);
  const size_t slots = 32 * size_t(b->Gpad);
  std::vector<uint32_t> perm(slots, 0u);
  std::vector<uint64_t> slot(2 * slots + b->Gpad, 0);
  for (size_t j = 0; j < n; ++j) {
    perm[j] = order[j];
    slot[j] = b->offsets[order[j]];
    slot[slots + j] = n_bits[order[j]];
  }
  for (uint32_t g = 0; g < b->G; ++g) {
    const uint64_t c = n_bits[order[size_t(g) * 32]];  // longest lane of the group
    slot[2 * slots + g] = c;
    b->group_clocks[g] = c;
    b->total_clocks += c;
    b->max_clocks = std::max(b->max_clocks, c);
  }
  bool ok = cudaMalloc(&b->d_in, 24 * n) == cudaSuccess &&
            cudaMalloc(&b->d_perm, slots * 4) == cudaSuccess &&
            cudaMalloc(&b->d_slot, slot.size() * 8) == cudaSuccess &&
            cudaMalloc(&b->d_state, size_t(kStateRows) * b->Gpad * 4) == cudaSuccess &&
            cudaMalloc(&b->d_scratch, size_t(kScratchRows + 1) * b->Gpad * 4) == cudaSuccess &&
            cudaMalloc(&b->d_queue, 8) == cudaSuccess &&
            cudaMalloc(&b->d_err, 4) == cudaSuccess &&
            cudaMalloc(&b->d_params, sizeof(BatchParams)) == cudaSuccess;
  if (ok) {
    std::vector<uint32_t> lens(n, 80u);
    if (iv_lens) std::copy(iv_lens, iv_lens + n, lens.begin());
    ok = cudaMemcpy(b->d_in + 20 * n, lens.data(), 4 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_perm, perm.data(), slots * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->d_slot, slot.data(), slot.size() * 8, cudaMemcpyHostToDevice) ==
             cudaSuccess &&
         cudaMemset(b->d_err, 0, 4) == cudaSuccess && capture(b) == cudaSuccess;
  }
  if (!ok) {
    batch_release(b);
    set_error(MICKEY_E_CUDA, "device allocation, upload or graph capture failed");
    return nullptr;
  }
  set_error(MICKEY_OK, "");
  return b;
}

MICKEY_API size_t mickey_batch_output_bytes(const mickey_batch *b) {
  return b ? size_t(b->out_bytes) : 0;
}

MICKEY_API int mickey_batch_offsets(const mickey_batch *b, uint64_t *offsets) {
  if (!b || !offsets) return set_error(MICKEY_E_ARG, "NULL argument");
  std::memcpy(offsets, b->offsets.data(), b->n * 8);
  return MICKEY_OK;
}

MICKEY_API int mickey_batch_clocks(const mickey_batch *b, uint64_t *max_clocks,
                                   uint64_t *total_clocks) {
  if (!b) return set_error(MICKEY_E_ARG, "NULL handle");
  if (max_clocks) *max_clocks = b->max_clocks;
  if (total_clocks) *total_clocks = b->total_clocks;
  return MICKEY_OK;
}

MICKEY_API int mickey_batch_run(mickey_batch *b, const void *keys, const void *ivs, void *out,
                                int mem) {
  if (!b || !keys || !ivs || !out) return set_error(MICKEY_E_ARG, "NULL argument");
  if (mem != MICKEY_MEM_HOST && mem != MICKEY_MEM_DEVICE)
    return set_error(MICKEY_E_ARG, "mem must be MICKEY_MEM_HOST or MICKEY_MEM_DEVICE");
  int rc = copy_inputs(b, keys, ivs, mem);
  if (rc) return rc;
  BatchParams p{static_cast<uint8_t *>(out)};
  if (cudaMemcpyAsync(b->d_params, &p, sizeof p, cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaGraphLaunch(b->exec, b->stream) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "graph launch");
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_batch_set_config(mickey_batch *b, int unroll, int blocks_per_sm,
                                       uint64_t split_clocks) {
  if (!b || !valid_unroll(unroll) || blocks_per_sm < 1 || blocks_per_sm > 2)
    return set_error(MICKEY_E_ARG, "unroll must be 2 or 4, blocks_per_sm 1 or 2");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(MICKEY_E_CUDA, "sync");
  b->unroll = unroll;
  b->blocks_per_sm = blocks_per_sm;
  b->split_clocks = split_clocks;
  uint32_t ns = 0;
  if (split_clocks)
    while (ns < b->G && b->group_clocks[ns] > split_clocks) ++ns;
  b->n_split = ns;
  return capture(b) == cudaSuccess ? MICKEY_OK : MICKEY_E_CUDA;
}

MICKEY_API int mickey_batch_set_split_mode(mickey_batch *b, int mode) {
  if (!b || (mode != MICKEY_BATCH_SPLIT_SHARED && mode != MICKEY_BATCH_SPLIT_OWN))
    return set_error(MICKEY_E_ARG, "split mode must be MICKEY_BATCH_SPLIT_SHARED or _OWN");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(MICKEY_E_CUDA, "sync");
  b->split_mode = mode;
  return capture(b) == cudaSuccess ? set_error(MICKEY_OK, "")
                                   : set_error(MICKEY_E_CUDA, "graph capture failed");
}

MICKEY_API int mickey_batch_get_split_mode(const mickey_batch *b) {
  if (!b) return set_error(MICKEY_E_ARG, "NULL handle");
  return b->split_mode;
}

MICKEY_API int mickey_batch_get_config(const mickey_batch *b, int *unroll, int *blocks_per_sm,
                                       uint64_t *split_clocks, uint32_t *split_groups) {
  if (!b || !unroll || !blocks_per_sm) return set_error(MICKEY_E_ARG, "NULL argument");
  *unroll = b->unroll;
  *blocks_per_sm = b->blocks_per_sm;
  if (split_clocks) *split_clocks = b->split_clocks;
  if (split_groups) *split_groups = b->n_split;
  return MICKEY_OK;
}

MICKEY_API int mickey_batch_sync(mickey_batch *b) {
  if (!b) return set_error(MICKEY_E_ARG, "NULL handle");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(MICKEY_E_CUDA, "sync");
  int flag = 0;
  if (cudaMemcpy(&flag, b->d_err, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "D2H err");
  if (flag) {
    cudaMemset(b->d_err, 0, 4);
    return (flag & kErrIvLen) ? set_error(MICKEY_E_IVLEN, "an IV length above 80 bits was given")
                              : set_error(MICKEY_E_TIMEOUT, "a device-side wait timed out");
  }
  return set_error(MICKEY_OK, "");
}

MICKEY_API void mickey_batch_free(mickey_batch *b) { batch_release(b); }

}  // extern "C"
