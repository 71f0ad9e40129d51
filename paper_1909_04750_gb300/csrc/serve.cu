// Serving: continuous batching over streams whose state stays resident on
// the device between requests.
//
// Stream table: one row of 8 words per stream -- R in words 0..3, S in
// words 4..7, register bit i at bit (31 - i % 32) of word i / 32 of its half.
// A step (one launch) takes a set of 32-lane groups chosen by the host
// scheduler: lane l of group g serves the request of stream slot_stream[..]
// and writes this step's keystream bytes at slot_out[..]; every lane of a
// group produces exactly group_clocks[g] bits (the host picks that as the
// smallest remaining length of the group's requests, capped by a quantum, so
// no request overshoots).  The kernel gathers each group's bitsliced state
// from the table, clocks it, and scatters it back.  Groups 0..n_split-1 (the
// longest remaining work) are clocked by a whole warp each (split path, a
// kernel of their own); the rest one group per thread, 32 groups per work
// item, from an atomic queue, in a second kernel after it on the stream.
#include <cuda_runtime.h>

#include <algorithm>

#include <cstring>
#include <new>
#include <vector>

#include "../../include/mickey.h"
#include "bitslice.cuh"
#include "internal.h"
#include "split.cuh"

using namespace mickey;

namespace {

constexpr int kServeThreads = 128;
constexpr uint32_t kNoStream = 0xffffffffu;

struct ServeArgs {
  uint32_t *packed;             // stream table [streams][8]
  const uint32_t *slot_stream;  // [32 * G]
  const uint64_t *slot_out;     // [32 * G] byte addresses (0: lane unused)
  const uint32_t *group_clocks; // [G]
  uint32_t G, n_split, n_items;
  uint32_t *queue;
};

// Bitsliced group state from the 32 lanes' table rows: for each 32-bit
// chunk q of the packed rows, a 32x32 transpose turns "row = lane" into
// "row = register bit".
__device__ __forceinline__ void gather_thread(const ServeArgs &a, uint32_t g, uint32_t (&r)[kReg],
                                              uint32_t (&s)[kReg]) {
  const uint32_t *ss = a.slot_stream + uint64_t(g) * 32;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int row = 0; row < 32; ++row) {
      const uint32_t st = ss[31 - row];
      m[row] = st != kNoStream ? a.packed[uint64_t(st) * 8 + q] : 0u;
    }
    transpose32(m);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int bit = 32 * (q & 3) + j;
      if (bit < kReg) {
        if (q < 4) r[bit] = m[j];
        else s[bit] = m[j];
      }
    }
  }
}

// Inverse of gather_thread.
__device__ __forceinline__ void scatter_thread(const ServeArgs &a, uint32_t g,
                                               const uint32_t (&r)[kReg],
                                               const uint32_t (&s)[kReg]) {
  const uint32_t *ss = a.slot_stream + uint64_t(g) * 32;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int bit = 32 * (q & 3) + j;
      m[j] = bit < kReg ? (q < 4 ? r[bit] : s[bit]) : 0u;
    }
    transpose32(m);  // m[31 - l]: lane l's chunk, register bit 32(q&3)+j at bit 31-j
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const uint32_t st = ss[l];
      if (st != kNoStream) a.packed[uint64_t(st) * 8 + q] = m[31 - l];
    }
  }
}

// Lane l's keystream bits of tile t (word in memory byte order), to its
// request buffer; whole bytes only (every step length is a multiple of 8).
__device__ __forceinline__ void store_lane(uint64_t base, uint32_t t, int nb, uint32_t w) {
  if (!base) return;
  uint8_t *o = reinterpret_cast<uint8_t *>(base) + 4ull * t;
  if (nb == 32 && (reinterpret_cast<uintptr_t>(o) & 3u) == 0) {
    *reinterpret_cast<uint32_t *>(o) = w;
  } else {
    const int nbytes = (nb + 7) >> 3;
    for (int b = 0; b < nbytes; ++b) o[b] = uint8_t(w >> (8 * b));
  }
}

// Un-bitslice a 32-clock tile held in shared memory (same two passes as the
// keystream kernels) and store each lane's word.
__device__ __forceinline__ void serve_emit(uint32_t *z, const ServeArgs &a, uint32_t g,
                                           uint32_t t, int nb) {
#pragma unroll 1
  for (int j = 0; j < 4; ++j) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = z[(8 * j + k) * kServeThreads];
    swap_bits<4>(v[0], v[4]); swap_bits<4>(v[1], v[5]);
    swap_bits<4>(v[2], v[6]); swap_bits<4>(v[3], v[7]);
    swap_bits<2>(v[0], v[2]); swap_bits<2>(v[1], v[3]);
    swap_bits<2>(v[4], v[6]); swap_bits<2>(v[5], v[7]);
    swap_bits<1>(v[0], v[1]); swap_bits<1>(v[2], v[3]);
    swap_bits<1>(v[4], v[5]); swap_bits<1>(v[6], v[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) z[(8 * j + k) * kServeThreads] = v[k];
  }
  const uint64_t *so = a.slot_out + uint64_t(g) * 32;
#pragma unroll 1
  for (int k = 0; k < 8; ++k) {
    uint32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = z[(k + 8 * q) * kServeThreads];
    swap_halves(v[0], v[2]);
    swap_halves(v[1], v[3]);
    swap_bytes<true>(v[0], v[1]);
    swap_bytes<true>(v[2], v[3]);
#pragma unroll
    for (int q = 0; q < 4; ++q) store_lane(so[31 - k - 8 * q], t, nb, v[q]);
  }
}

template <int U>
__device__ __forceinline__ void serve_group(const ServeArgs &a, uint32_t g, uint32_t *z) {
  uint32_t r[kReg], s[kReg];
  gather_thread(a, g, r, s);
  const uint32_t clocks = a.group_clocks[g];
  const uint32_t full = clocks >> 5;
#pragma unroll 1
  for (uint32_t tile = 0; tile < full; ++tile) {
#pragma unroll 1
    for (int c = 0; c < 32; c += U) {
#pragma unroll
      for (int u = 0; u < U; ++u) {
        z[(c + u) * kServeThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      }
    }
    serve_emit(z, a, g, tile, 32);
  }
  const int rem = int(clocks & 31);
  if (rem) {
#pragma unroll 1
    for (int c = 0; c < 32; ++c) {
      if (c < rem) {
        z[c * kServeThreads] = r[0] ^ s[0];
        clock_kg<false, false>(r, s, 0u, 0u);
      } else {
        z[c * kServeThreads] = 0u;
      }
    }
    serve_emit(z, a, g, full, rem);
  }
  scatter_thread(a, g, r, s);
}

// Split path: lane l brings its stream's row; 200 ballots give each lane
// the bitsliced words of its slots (R bit 4j+q, S bit 100-4j-q).
__device__ __forceinline__ void serve_split(const ServeArgs &a, uint32_t g, uint32_t lane,
                                            uint32_t *zbuf0, uint32_t *zbuf1) {
  const uint32_t st = a.slot_stream[uint64_t(g) * 32 + lane];
  uint32_t row[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) row[q] = st != kNoStream ? a.packed[uint64_t(st) * 8 + q] : 0u;
  uint32_t r[4] = {0, 0, 0, 0}, s[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    const uint32_t wr = __ballot_sync(0xffffffffu, (row[i >> 5] >> (31 - (i & 31))) & 1u);
    const uint32_t ws = __ballot_sync(0xffffffffu, (row[4 + (i >> 5)] >> (31 - (i & 31))) & 1u);
    if (lane == uint32_t(i >> 2)) r[i & 3] = wr;
    if (lane == uint32_t((100 - i) >> 2)) s[(100 - i) & 3] = ws;
  }
  SplitLane k;
  split_lane_init(lane, k);
  const uint64_t base = a.slot_out[uint64_t(g) * 32 + lane];
  const uint32_t clocks = a.group_clocks[g];
  const uint32_t full = clocks >> 5;
#pragma unroll 1
  for (uint32_t t = 0; t < full; ++t) {
    const uint32_t mine = split_tile<kSplitUnroll>(r, s, k, lane, zbuf0, zbuf1, 32);
    store_lane(base, t, 32, __byte_perm(__brev(mine), 0u, 0x0123));
  }
  const int rem = int(clocks & 31);
  if (rem) {
    const uint32_t mine = split_tile<kSplitUnroll>(r, s, k, lane, zbuf0, zbuf1, rem);
    store_lane(base, full, rem, __byte_perm(__brev(mine), 0u, 0x0123));
  }
  // back to rows
  uint32_t out[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    const uint32_t xr = __shfl_sync(0xffffffffu, r[i & 3], i >> 2);
    const uint32_t xs = __shfl_sync(0xffffffffu, s[(100 - i) & 3], (100 - i) >> 2);
    out[i >> 5] |= ((xr >> lane) & 1u) << (31 - (i & 31));
    out[4 + (i >> 5)] |= ((xs >> lane) & 1u) << (31 - (i & 31));
  }
  if (st != kNoStream) {
#pragma unroll
    for (int q = 0; q < 8; ++q) a.packed[uint64_t(st) * 8 + q] = out[q];
  }
}

// One group per thread, 32 groups per work item, from the atomic queue.
template <int U>
__global__ void __launch_bounds__(kServeThreads) serve_step_kernel(ServeArgs a) {
  __shared__ uint32_t zs[32 * kServeThreads];
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    const uint32_t g = item * 32 + lane;
    if (g < a.G) serve_group<U>(a, g, zs + threadIdx.x);
  }
}

// Split groups only (a step's groups 0 .. n_split-1), with a register
// budget of its own: the one-thread-per-group path needs the whole register
// file of a thread, which limits a combined kernel to 2 warps per SM
// sub-partition; this one runs at least 4.
constexpr int kSplitMinBlocksPerSm = 4;
__global__ void __launch_bounds__(kServeThreads, kSplitMinBlocksPerSm)
    serve_split_kernel(ServeArgs a) {
  __shared__ uint32_t zs[2 * kServeThreads];   // 2 x 32 words per warp
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll 1
  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(a.queue, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_split) break;
    uint32_t *zb = zs + (threadIdx.x & ~31u);
    serve_split(a, item, lane, zb, zb + kServeThreads);
  }
}

// Initial states (word-major bitsliced, as written by the preclock kernel)
// to table rows.
__global__ void __launch_bounds__(kServeThreads)
    pack_states_kernel(const uint32_t *state, uint32_t G, uint32_t Gpad,
                       const uint32_t *slot_stream, uint32_t *packed) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
#pragma unroll 1
  for (int q = 0; q < 8; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int bit = 32 * (q & 3) + j;
      m[j] = bit < kReg ? state[size_t((q < 4 ? 0 : kReg) + bit) * Gpad + g] : 0u;
    }
    transpose32(m);
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const uint32_t st = slot_stream[uint64_t(g) * 32 + l];
      if (st != kNoStream) packed[uint64_t(st) * 8 + q] = m[31 - l];
    }
  }
}

}  // namespace

struct mickey_server {
  size_t max_streams = 0;
  uint32_t max_groups = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0, unroll = 4, blocks_per_sm = 2, split_blocks_per_sm = kSplitMinBlocksPerSm;
  uint32_t *d_packed = nullptr;
  // per-step metadata, double buffered: slot_stream, slot_out, group_clocks, queue
  struct Meta {
    uint32_t *d_stream = nullptr;
    uint64_t *d_out = nullptr;
    uint32_t *d_clocks = nullptr, *d_queue = nullptr;
    void *h_stage = nullptr;   // pinned host staging of the three arrays
    cudaEvent_t done = nullptr;
  } meta[2];
  int cur = 0;
  // init of new streams
  mickey_streams *init = nullptr;
  size_t init_cap = 0;
  uint32_t *d_init_slots = nullptr;
};

namespace {

void server_release(mickey_server *s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto &m : s->meta) {
    cudaFree(m.d_stream);
    cudaFree(m.d_out);
    cudaFree(m.d_clocks);
    cudaFree(m.d_queue);
    if (m.h_stage) cudaFreeHost(m.h_stage);
    if (m.done) cudaEventDestroy(m.done);
  }
  cudaFree(s->d_packed);
  cudaFree(s->d_init_slots);
  if (s->init) mickey_free(s->init);
  delete s;
}

size_t meta_bytes(uint32_t groups) { return size_t(groups) * 32 * (4 + 8) + size_t(groups) * 4; }

}  // namespace

extern "C" {

MICKEY_API mickey_server *mickey_server_create(size_t max_streams, uint32_t max_groups,
                                               void *cuda_stream) {
  if (max_streams == 0 || max_streams >= kNoStream || max_groups == 0) {
    set_error(MICKEY_E_ARG, "need 0 < max_streams < 2^32 - 1 and max_groups > 0");
    return nullptr;
  }
  mickey_server *s = new (std::nothrow) mickey_server;
  if (!s) {
    set_error(MICKEY_E_OOM, "host allocation failed");
    return nullptr;
  }
  s->max_streams = max_streams;
  s->max_groups = max_groups;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev);
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, serve_split_kernel, kServeThreads, 0) ==
          cudaSuccess &&
      nb > 0)
    s->split_blocks_per_sm = nb;
  bool ok = cudaMalloc(&s->d_packed, max_streams * 32) == cudaSuccess &&
            cudaMemset(s->d_packed, 0, max_streams * 32) == cudaSuccess;
  for (auto &m : s->meta) {
    ok = ok && cudaMalloc(&m.d_stream, size_t(max_groups) * 32 * 4) == cudaSuccess &&
         cudaMalloc(&m.d_out, size_t(max_groups) * 32 * 8) == cudaSuccess &&
         cudaMalloc(&m.d_clocks, size_t(max_groups) * 4) == cudaSuccess &&
         cudaMalloc(&m.d_queue, 8) == cudaSuccess &&
         cudaMallocHost(&m.h_stage, meta_bytes(max_groups)) == cudaSuccess &&
         cudaEventCreateWithFlags(&m.done, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    server_release(s);
    set_error(MICKEY_E_OOM, "server allocation failed");
    return nullptr;
  }
  set_error(MICKEY_OK, "");
  return s;
}

// Load and preclock n new streams and write their states to table rows
// stream_ids[i].  Host inputs.
MICKEY_API int mickey_server_init_streams(mickey_server *s, const uint32_t *stream_ids,
                                          const uint8_t *keys, const uint8_t *ivs,
                                          const uint32_t *iv_lens, size_t n) {
  if (!s || !stream_ids || !keys || !ivs) return set_error(MICKEY_E_ARG, "NULL argument");
  if (n == 0) return set_error(MICKEY_OK, "");
  for (size_t i = 0; i < n; ++i)
    if (stream_ids[i] >= s->max_streams)
      return set_error(MICKEY_E_ARG, "stream id beyond the table");
  if (n > s->init_cap) {
    if (s->init) mickey_free(s->init);
    s->init = nullptr;
    cudaFree(s->d_init_slots);
    s->d_init_slots = nullptr;
    s->init_cap = 0;
  }
  std::vector<uint32_t> slots(((n + 31) / 32) * 32, kNoStream);
  std::memcpy(slots.data(), stream_ids, n * 4);
  if (!s->init) {
    s->init = mickey_init_streams_ex(keys, ivs, iv_lens, n, MICKEY_MEM_HOST, s->stream);
    if (!s->init) return mickey_last_error();
    if (cudaMalloc(&s->d_init_slots, slots.size() * 4) != cudaSuccess)
      return set_error(MICKEY_E_OOM, "init slots");
    s->init_cap = n;
  } else {
    // same handle size is required by reset: pad to the handle's n
    const size_t cap = mickey_num_streams(s->init);
    std::vector<uint8_t> k(cap * 10, 0), v(cap * 10, 0);
    std::vector<uint32_t> l(cap, 80);
    std::memcpy(k.data(), keys, n * 10);
    std::memcpy(v.data(), ivs, n * 10);
    if (iv_lens) std::memcpy(l.data(), iv_lens, n * 4);
    const int rc = mickey_reset_streams(s->init, k.data(), v.data(), l.data(), MICKEY_MEM_HOST);
    if (rc) return rc;
  }
  if (cudaMemcpyAsync(s->d_init_slots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice,
                      s->stream) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "init slots upload");
  uint32_t G = 0, Gpad = 0;
  const uint32_t *state = handle_state(s->init, &G, &Gpad);
  const uint32_t Gn = uint32_t((n + 31) / 32);
  pack_states_kernel<<<(Gn + kServeThreads - 1) / kServeThreads, kServeThreads, 0, s->stream>>>(
      state, Gn, Gpad, s->d_init_slots, s->d_packed);
  if (cudaGetLastError() != cudaSuccess) return set_error(MICKEY_E_CUDA, "pack kernel");
  // every upload above is stream-ordered, so the next call may reuse the
  // handle and the slot list without waiting here
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_server_step(mickey_server *s, uint32_t G, uint32_t n_split,
                                  const uint32_t *slot_stream, const uint64_t *slot_out,
                                  const uint32_t *group_clocks) {
  if (!s || !slot_stream || !slot_out || !group_clocks)
    return set_error(MICKEY_E_ARG, "NULL argument");
  if (G == 0) return set_error(MICKEY_OK, "");
  if (G > s->max_groups || n_split > G) return set_error(MICKEY_E_ARG, "too many groups");
  for (size_t i = 0; i < size_t(G) * 32; ++i)
    if (slot_stream[i] != kNoStream && slot_stream[i] >= s->max_streams)
      return set_error(MICKEY_E_ARG, "stream id beyond the table");
  auto &m = s->meta[s->cur];
  s->cur ^= 1;
  // the staging of this buffer set was last used two steps ago
  if (cudaEventSynchronize(m.done) != cudaSuccess) return set_error(MICKEY_E_CUDA, "event");
  uint8_t *h = static_cast<uint8_t *>(m.h_stage);
  const size_t ns = size_t(G) * 32 * 4, no = size_t(G) * 32 * 8, nc = size_t(G) * 4;
  std::memcpy(h, slot_stream, ns);
  std::memcpy(h + ns, slot_out, no);
  std::memcpy(h + ns + no, group_clocks, nc);
  if (cudaMemcpyAsync(m.d_stream, h, ns, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(m.d_out, h + ns, no, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemcpyAsync(m.d_clocks, h + ns + no, nc, cudaMemcpyHostToDevice, s->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(m.d_queue, 0, 8, s->stream) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "step upload");
  // split groups: their own kernel, up to 4 warps per SM sub-partition
  if (n_split) {
    ServeArgs a{s->d_packed, m.d_stream, m.d_out, m.d_clocks, n_split, n_split, n_split,
                m.d_queue};
    const uint32_t warps = kServeThreads / 32;
    const uint32_t grid = std::min<uint32_t>((n_split + warps - 1) / warps,
                                             uint32_t(s->sm_count * s->split_blocks_per_sm));
    serve_split_kernel<<<grid, kServeThreads, 0, s->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return set_error(MICKEY_E_CUDA, "split kernel");
  }
  // the rest one group per thread, after them on the stream
  if (G > n_split) {
    const uint32_t Gt = G - n_split;
    ServeArgs a{s->d_packed, m.d_stream + size_t(n_split) * 32, m.d_out + size_t(n_split) * 32,
                m.d_clocks + n_split, Gt, 0, (Gt + 31) / 32, m.d_queue + 1};
    const uint32_t grid = uint32_t(s->sm_count * s->blocks_per_sm);
    if (s->unroll == 2)
      serve_step_kernel<2><<<grid, kServeThreads, 0, s->stream>>>(a);
    else
      serve_step_kernel<4><<<grid, kServeThreads, 0, s->stream>>>(a);
    if (cudaGetLastError() != cudaSuccess) return set_error(MICKEY_E_CUDA, "step kernel");
  }
  if (cudaEventRecord(m.done, s->stream) != cudaSuccess) return set_error(MICKEY_E_CUDA, "event");
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_server_read_states(mickey_server *s, const uint32_t *stream_ids, size_t n,
                                         uint8_t *states) {
  if (!s || !stream_ids || !states) return set_error(MICKEY_E_ARG, "NULL argument");
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return set_error(MICKEY_E_CUDA, "sync");
  for (size_t i = 0; i < n; ++i) {
    if (stream_ids[i] >= s->max_streams) return set_error(MICKEY_E_ARG, "stream id");
    uint32_t row[8];
    if (cudaMemcpy(row, s->d_packed + uint64_t(stream_ids[i]) * 8, 32, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return set_error(MICKEY_E_CUDA, "D2H");
    uint8_t *rec = states + 26 * i;
    std::memset(rec, 0, 26);
    for (int half = 0; half < 2; ++half)
      for (int b = 0; b < kReg; ++b)
        if ((row[4 * half + b / 32] >> (31 - b % 32)) & 1u)
          rec[13 * half + b / 8] |= uint8_t(0x80u >> (b % 8));
  }
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_server_set_config(mickey_server *s, int unroll, int blocks_per_sm) {
  if (!s || (unroll != 2 && unroll != 4) || blocks_per_sm < 1 || blocks_per_sm > 2)
    return set_error(MICKEY_E_ARG, "unroll 2 or 4, blocks_per_sm 1 or 2");
  s->unroll = unroll;
  s->blocks_per_sm = blocks_per_sm;
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_server_sync(mickey_server *s) {
  if (!s) return set_error(MICKEY_E_ARG, "NULL handle");
  return cudaStreamSynchronize(s->stream) == cudaSuccess ? set_error(MICKEY_OK, "")
                                                          : set_error(MICKEY_E_CUDA, "sync");
}

MICKEY_API void mickey_server_free(mickey_server *s) { server_release(s); }

}  // extern "C"
