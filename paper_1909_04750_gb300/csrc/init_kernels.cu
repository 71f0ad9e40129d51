// Key/IV loading and preclocking for bitsliced MICKEY 2.0 (Sec. IV-A
// representation change, Sec. IV-D input handler, and the cipher's
// initialisation), in one kernel: one thread per 32-lane group.
//
// Load    the group's 32 keys, IVs and IV lengths become bitsliced words by
//         32x32 bit-matrix transposes (row-major -> column-major, Sec. IV-A),
//         written to the group's column of the scratch rows.  IVs are
//         right-aligned per lane so that all lanes of a group end their IV
//         phase on the same clock; a lane with a shorter IV is held still
//         (masked) until its first IV bit.
// Preclock zero state, IV clocks, 80 key clocks, 100 mixing preclocks, all
//         in mixing mode, reading the scratch words the same thread has just
//         written; writes the 200-word state.
// In one launch the loading of some warps (memory latency) overlaps the
// clocking of others (logic issue).  When the instances are in their own
// order (no permutation) and 16-byte aligned, each thread reads its 32
// lanes' records with 16-byte loads into registers; unaligned, a block first
// copies its 32 x kInitThreads keys, IVs and IV lengths into shared memory
// with coalesced 4-byte cp.async copies; permuted, each lane's record is read
// byte by byte.
#include "bitslice.cuh"
#include "internal.h"

namespace mickey {
namespace {

__device__ __forceinline__ uint32_t load_be32(const uint8_t *p) {
  return (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16) |
         (uint32_t(p[2]) << 8) | uint32_t(p[3]);
}

// Word k (k = 0 most significant) of the mask selecting the first m bits
// of a 96-bit big-endian bit string.
__device__ __forceinline__ uint32_t prefix_mask(int m, int k) {
  const int lo = 32 * k;
  if (m >= lo + 32) return ~0u;
  if (m <= lo) return 0u;
  return ~0u << (32 - (m - lo));
}

__device__ __forceinline__ uint32_t pick3(uint32_t w0, uint32_t w1,
                                          uint32_t w2, int idx) {
  return idx == 0 ? w0 : idx == 1 ? w1 : idx == 2 ? w2 : 0u;
}

// Word k of the 96-bit big-endian string (w0, w1, w2) moved s bits towards
// higher bit indices (bit b -> bit b + s); 0 <= s <= 80.
__device__ __forceinline__ uint32_t shift96_word(uint32_t w0, uint32_t w1,
                                                 uint32_t w2, int s, int k) {
  const int ws = s >> 5, bs = s & 31;
  const int i_lo = k - ws, i_hi = k - ws - 1;
  const uint32_t lo = i_lo >= 0 ? pick3(w0, w1, w2, i_lo) : 0u;
  const uint32_t hi = i_hi >= 0 ? pick3(w0, w1, w2, i_hi) : 0u;
  return __funnelshift_r(lo, hi, bs);
}

// Shared-memory staging of a block's inputs (instances in their own order):
// thread t's 32 ten-byte keys as words 81t .. 81t+79 (one spare word, so
// that the rows of a warp's threads start in different banks), the same for
// the IVs, and its 32 IV lengths at 33t .. 33t+31.
constexpr int kRecWords = 81;
constexpr int kLenWords = 33;
constexpr size_t kStageBytes = size_t(kInitThreads) * (2 * kRecWords + kLenWords) * 4;

// Big-endian 32 bits at byte offset o of a staged 320-byte row (the bytes
// past the row's end come from the spare word or the next row and are masked
// off by the caller).
__device__ __forceinline__ uint32_t staged_be32(const uint32_t *row, int o) {
  const uint32_t w0 = row[o >> 2], w1 = row[(o >> 2) + 1];
  return __byte_perm(__funnelshift_r(w0, w1, 8 * (o & 3)), 0u, 0x0123);
}

// Where one group's inputs come from: the staged rows of its thread, or
// global memory (through the permutation, if any).
struct Src {
  const LoadArgs *a;
  uint64_t base;          // slot of lane 0
  const uint32_t *krow;   // staged: 80 key words of this thread (else nullptr)
  const uint32_t *vrow;   // staged IV words
  const uint32_t *lrow;   // staged IV lengths
  __device__ uint64_t inst(int l) const {
    return a->perm ? uint64_t(a->perm[base + l]) : base + l;
  }
  // chunk q (q = 0, 1: 32 bits; q = 2: the last 16 bits, in the high half)
  // of lane l's key or IV, big-endian
  __device__ uint32_t chunk(bool iv, int l, int q) const {
    if (krow) {
      const uint32_t v = staged_be32(iv ? vrow : krow, 10 * l + 4 * q);
      return q < 2 ? v : v & 0xFFFF0000u;
    }
    const uint8_t *p = (iv ? a->ivs : a->keys) + inst(l) * 10 + 4 * q;
    return q < 2 ? load_be32(p) : (uint32_t(p[0]) << 24) | (uint32_t(p[1]) << 16);
  }
  __device__ uint32_t iv_len(int l) const {
    if (lrow) return lrow[l];
    return a->iv_lens ? a->iv_lens[inst(l)] : 80u;
  }
};

// The load of group g: bitsliced key rows, right-aligned IV rows, activity
// rows (mixed IV lengths only) and the info word.
__device__ __forceinline__ void load_group(const LoadArgs &a, uint32_t g, const Src &src) {
  const uint64_t base = 32ull * g;
  const uint64_t left = a.n - base;
  const int nv = left >= 32 ? 32 : int(left);

  int len[32];
  int max_len = 0, min_len = 80;
#pragma unroll
  for (int l = 0; l < 32; ++l) {
    int v = 0;
    if (l < nv) {
      v = int(min(src.iv_len(l), 1000u));
      if (v > 80) {
        atomicOr(a.err, kErrIvLen);
        v = 80;
      }
      max_len = max(max_len, v);
      min_len = min(min_len, v);
    }
    len[l] = v;
  }
  // The IV phase runs a multiple of 4 clocks (the preclock loop handles four
  // clocks per iteration); lanes are right-aligned to that length.
  const int phase = (max_len + 3) & ~3;
#pragma unroll
  for (int l = 0; l < 32; ++l)
    if (l >= nv) len[l] = phase;  // padding lanes: zero inputs, no masking
  const bool mixed = min_len != phase;

  // Key bits: three 32-bit chunks per lane (the third holds bits 64..79).
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;  // row r = lane 31-r, so result bit l = lane l
      m[r] = l < nv ? src.chunk(false, l, q) : 0u;
    }
    transpose32(m);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int row = 32 * q + j;
      if (row < 80) a.scratch[size_t(kKeyRow + row) * a.Gpad + g] = m[j];
    }
  }

  // IV bits, right-aligned: lane l's bit b is consumed at IV clock
  // b + (phase - len[l]); before that the lane is inactive (zero state).
#pragma unroll 1
  for (int q = 0; q < 3; ++q) {
    if (32 * q >= phase) break;
    uint32_t m[32], act[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const int l = 31 - r;
      const int L = len[l];
      const int sft = phase - L;
      uint32_t w = 0;
      if (l < nv && L > 0) {
        const uint32_t w0 = src.chunk(true, l, 0) & prefix_mask(L, 0);
        const uint32_t w1 = src.chunk(true, l, 1) & prefix_mask(L, 1);
        const uint32_t w2 = src.chunk(true, l, 2) & prefix_mask(L, 2);
        w = shift96_word(w0, w1, w2, sft, q);
      }
      m[r] = w;
      act[r] = prefix_mask(phase, q) & ~prefix_mask(sft, q);
    }
    transpose32(m);
    if (mixed) transpose32(act);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = 32 * q + j;
      if (c < phase) {
        a.scratch[size_t(kIvRow + c) * a.Gpad + g] = m[j];
        if (mixed) a.scratch[size_t(kActRow + c) * a.Gpad + g] = act[j];
      }
    }
  }
  a.scratch[size_t(kScratchRows) * a.Gpad + g] = uint32_t(phase) | (mixed ? 0x100u : 0u);
}

// The load of a whole group (32 instances) whose keys, IVs and IV lengths
// are 16-byte aligned in their own order: each thread reads its 32 records
// (320 bytes of keys, the same of IVs, 128 bytes of lengths) with 16-byte
// loads, all in flight at once, and cuts every lane's chunks out of the
// words at byte offsets known at compile time.  Same result as load_group.
__device__ __forceinline__ void load_records(const uint8_t *base, uint32_t (&w)[80]) {
  const uint4 *p = reinterpret_cast<const uint4 *>(base);
#pragma unroll
  for (int i = 0; i < 20; ++i) {
    const uint4 x = __ldg(p + i);
    w[4 * i] = x.x;
    w[4 * i + 1] = x.y;
    w[4 * i + 2] = x.z;
    w[4 * i + 3] = x.w;
  }
}

// Chunk q of lane l's record (as Src::chunk) from the words of load_records:
// the byte offset 10l + 4q is even, so a chunk starts at byte 0 or 2 of a word.
__device__ __forceinline__ uint32_t record_chunk(const uint32_t (&w)[80], int l, int q) {
  const int o = 10 * l + 4 * q, i = o >> 2;
  uint32_t x;
  if (q < 2)
    x = (o & 2) ? __funnelshift_r(w[i], w[i + 1], 16) : w[i];
  else
    x = (o & 2) ? (w[i] >> 16) : (w[i] & 0xFFFFu);
  const uint32_t be = __byte_perm(x, 0u, 0x0123);
  return q < 2 ? be : be & 0xFFFF0000u;
}

__device__ __forceinline__ void load_group_regs(const LoadArgs &a, uint32_t g) {
  int len[32];
  int max_len = 80, min_len = 80;
  if (a.iv_lens) {
    const uint4 *lp = reinterpret_cast<const uint4 *>(a.iv_lens + 32ull * g);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const uint4 x = __ldg(lp + i);
      len[4 * i] = int(min(x.x, 1000u));
      len[4 * i + 1] = int(min(x.y, 1000u));
      len[4 * i + 2] = int(min(x.z, 1000u));
      len[4 * i + 3] = int(min(x.w, 1000u));
    }
    max_len = 0;
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      if (len[l] > 80) {
        atomicOr(a.err, kErrIvLen);
        len[l] = 80;
      }
      max_len = max(max_len, len[l]);
      min_len = min(min_len, len[l]);
    }
  } else {
#pragma unroll
    for (int l = 0; l < 32; ++l) len[l] = 80;
  }
  const int phase = (max_len + 3) & ~3;
  const bool mixed = min_len != phase;
  const size_t P = a.Gpad;

  uint32_t w[80];
  load_records(a.keys + 320ull * g, w);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    uint32_t m[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) m[r] = record_chunk(w, 31 - r, q);  // row r = lane 31-r
    transpose32(m);
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (32 * q + j < 80) a.scratch[size_t(kKeyRow + 32 * q + j) * P + g] = m[j];
  }

  load_records(a.ivs + 320ull * g, w);
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (32 * q < phase) {
      uint32_t m[32];
      if (!mixed) {  // every lane's IV fills the whole phase: no shift, no mask rows
        const uint32_t pm = prefix_mask(phase, q);
#pragma unroll
        for (int r = 0; r < 32; ++r) m[r] = record_chunk(w, 31 - r, q) & pm;
        transpose32(m);
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (32 * q + j < phase) a.scratch[size_t(kIvRow + 32 * q + j) * P + g] = m[j];
      } else {
        uint32_t act[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          const int l = 31 - r, L = len[l], sft = phase - L;
          const uint32_t c0 = record_chunk(w, l, 0) & prefix_mask(L, 0);
          const uint32_t c1 = record_chunk(w, l, 1) & prefix_mask(L, 1);
          const uint32_t c2 = record_chunk(w, l, 2) & prefix_mask(L, 2);
          m[r] = L > 0 ? shift96_word(c0, c1, c2, sft, q) : 0u;
          act[r] = prefix_mask(phase, q) & ~prefix_mask(sft, q);
        }
        transpose32(m);
        transpose32(act);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = 32 * q + j;
          if (c < phase) {
            a.scratch[size_t(kIvRow + c) * P + g] = m[j];
            a.scratch[size_t(kActRow + c) * P + g] = act[j];
          }
        }
      }
    }
  }
  a.scratch[size_t(kScratchRows) * P + g] = uint32_t(phase) | (mixed ? 0x100u : 0u);
}

constexpr int kPre = 4;  // clocks per loop iteration (IV phases and 180 are multiples of 4)

// Group g's state after initialisation, left in r and s: zero state, the IV
// clocks, 80 key clocks and 100 preclocks, every clock in mixing mode, from
// the scratch rows the loading has just written (kScratchRows rows of P
// words, then the info word per group: IV clocks | mixed << 8).  kPre clocks
// per loop iteration: with a single clock per iteration the shift of both
// registers makes every loop-carried word change register, which costs
// copies and spills; four clocks with the input rows read two iterations
// ahead took the whole kernel from 266 to 211 us for 2^20 instances and from
// 3.16 to 2.50 ms for 2^24 (with the 16-byte loads below).  The IV (unless
// lanes are masked), key and preclock phases share one loop body, the
// clock's input word chosen by its index: one copy of the clock's code, so
// that warps in different phases fetch the same instructions.
__device__ __forceinline__ void preclock_regs(const uint32_t *rows, size_t P, uint32_t g,
                                              uint32_t (&r)[kReg], uint32_t (&s)[kReg]) {
#pragma unroll
  for (int i = 0; i < kReg; ++i) r[i] = s[i] = 0u;

  const uint32_t info = rows[size_t(kScratchRows) * P + g];
  const int phase = int(info & 0xFFu);  // IV clocks, a multiple of 4
  const bool mixed = (info >> 8) & 1u;
  const uint32_t *col = rows + g;

  // Each loop reads its input rows two iterations ahead, so that the loads
  // are in flight while the clocks before them run.
  int c0 = 0;
  if (mixed) {
    uint32_t v[2 * kPre], m[2 * kPre];
#pragma unroll
    for (int u = 0; u < 2 * kPre; ++u) {
      const int cc = u < phase ? u : 0;
      v[u] = col[(kIvRow + cc) * P];
      m[u] = col[(kActRow + cc) * P];
    }
#pragma unroll 1
    for (int c = 0; c < phase; c += kPre) {
      uint32_t cv[kPre], cm[kPre];
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        cv[u] = v[u];
        cm[u] = m[u];
        v[u] = v[kPre + u];
        m[u] = m[kPre + u];
        const int cc = c + 2 * kPre + u < phase ? c + 2 * kPre + u : 0;
        v[kPre + u] = col[(kIvRow + cc) * P];
        m[kPre + u] = col[(kActRow + cc) * P];
      }
#pragma unroll
      for (int u = 0; u < kPre; ++u) clock_kg<true, true>(r, s, cv[u], cm[u]);
    }
    c0 = phase;
  }
  // clock c: IV bit c (c < phase), key bit c - phase (c < phase + 80), else
  // 0; one load per clock, of row 0 when the clock takes no input
  const int end = phase + 180;
  auto row_of = [phase](int c) {
    return c >= phase + 80 ? 0 : c < phase ? kIvRow + c : kKeyRow + c - phase;
  };
  uint32_t v[2 * kPre];
#pragma unroll
  for (int u = 0; u < 2 * kPre; ++u) v[u] = col[size_t(row_of(c0 + u)) * P];
#pragma unroll 1
  for (int c = c0; c < end; c += kPre) {
    uint32_t cv[kPre];
#pragma unroll
    for (int u = 0; u < kPre; ++u) {
      cv[u] = v[u];
      v[u] = v[kPre + u];
      v[kPre + u] = col[size_t(row_of(c + 2 * kPre + u)) * P];
    }
#pragma unroll
    for (int u = 0; u < kPre; ++u)
      clock_kg<true, false>(r, s, c + u < phase + 80 ? cv[u] : 0u, 0u);
  }
}

// The preclock of group g from its scratch column (written by this
// thread), stored as the group's 200 state words.
__device__ __forceinline__ void preclock_group(const LoadArgs &a, uint32_t *state, uint32_t g) {
  uint32_t r[kReg], s[kReg];
  preclock_regs(a.scratch, a.Gpad, g, r, s);
  uint32_t *st = state + g;
  const size_t P = a.Gpad;
#pragma unroll
  for (int i = 0; i < kReg; ++i) {
    st[size_t(i) * P] = r[i];
    st[size_t(kReg + i) * P] = s[i];
  }
}

// Copy `bytes` bytes from global src to the staged rows at dst: byte b of
// the source goes to row b / row_bytes, offset b % row_bytes, rows
// stride_words apart.  When src is 4-byte aligned the words go by cp.async
// (global to shared without a register round trip, all of a thread's copies
// in flight at once; the caller waits for them); otherwise byte loads.
__device__ __forceinline__ void stage_rows(const uint8_t *src, uint64_t bytes, uint32_t *dst,
                                           int row_bytes, int stride_words) {
  const uint32_t t = threadIdx.x;
  const int row_words = row_bytes / 4;
  if ((reinterpret_cast<uintptr_t>(src) & 3u) == 0) {
    const uint32_t *s4 = reinterpret_cast<const uint32_t *>(src);
    const uint64_t words = bytes / 4;
    for (uint64_t w = t; w < words; w += kInitThreads) {
      const uint32_t d = uint32_t(__cvta_generic_to_shared(
          dst + (w / row_words) * stride_words + w % row_words));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(s4 + w) : "memory");
    }
    // a last partial word (byte copies into the row's word)
    if (t == 0 && (bytes & 3)) {
      uint32_t v = 0;
      for (uint64_t b = words * 4; b < bytes; ++b) v |= uint32_t(src[b]) << (8 * (b & 3));
      dst[(words / row_words) * stride_words + words % row_words] = v;
    }
  } else {
    for (uint64_t w = t; w * 4 < bytes; w += kInitThreads) {
      uint32_t v = 0;
      for (int b = 0; b < 4 && w * 4 + b < bytes; ++b) v |= uint32_t(src[w * 4 + b]) << (8 * b);
      dst[(w / row_words) * stride_words + w % row_words] = v;
    }
  }
}

// Where the loading reads the inputs from: global memory byte by byte
// (through the permutation, if any), the block's shared-memory copy, or
// 16-byte loads into registers (aligned inputs in their own order; the last
// group, if partial, reads byte by byte).
enum SrcKind { kSrcGlobal, kSrcStaged, kSrcRegs };

template <int SRC>
__global__ void __launch_bounds__(kInitThreads) init_kernel(LoadArgs a, uint32_t *state) {
  extern __shared__ uint32_t stage[];
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  Src src{&a, 32ull * g, nullptr, nullptr, nullptr};
  if constexpr (SRC == kSrcStaged) {
    // the block's instances, in their own order: keys, IVs, IV lengths
    const uint64_t first = 32ull * blockIdx.x * kInitThreads;
    const uint64_t count = min(uint64_t(32) * kInitThreads, a.n - first);
    uint32_t *ks = stage, *vs = stage + kInitThreads * kRecWords;
    uint32_t *ls = vs + kInitThreads * kRecWords;
    stage_rows(a.keys + first * 10, count * 10, ks, 320, kRecWords);
    stage_rows(a.ivs + first * 10, count * 10, vs, 320, kRecWords);
    if (a.iv_lens)
      stage_rows(reinterpret_cast<const uint8_t *>(a.iv_lens + first), count * 4, ls, 128,
                 kLenWords);
    else
      for (uint32_t i = threadIdx.x; i < kInitThreads * kLenWords; i += kInitThreads) ls[i] = 80u;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    src.krow = ks + threadIdx.x * kRecWords;
    src.vrow = vs + threadIdx.x * kRecWords;
    src.lrow = ls + threadIdx.x * kLenWords;
  }
  if (g >= a.G) return;
  if (SRC == kSrcRegs && 32ull * g + 32 <= a.n)
    load_group_regs(a, g);
  else
    load_group(a, g, src);
  preclock_group(a, state, g);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

cudaError_t launch_init(const LoadArgs &a, uint32_t *state, cudaStream_t st) {
  const uint32_t blocks = (a.G + kInitThreads - 1) / kInitThreads;
  if (!a.perm && aligned16(a.keys) && aligned16(a.ivs) && (!a.iv_lens || aligned16(a.iv_lens))) {
    init_kernel<kSrcRegs><<<blocks, kInitThreads, 0, st>>>(a, state);
  } else if (a.perm) {
    init_kernel<kSrcGlobal><<<blocks, kInitThreads, 0, st>>>(a, state);
  } else {
    const cudaError_t e = cudaFuncSetAttribute(
        init_kernel<kSrcStaged>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStageBytes));
    if (e != cudaSuccess) return e;
    init_kernel<kSrcStaged><<<blocks, kInitThreads, kStageBytes, st>>>(a, state);
  }
  return cudaGetLastError();
}

}  // namespace mickey
