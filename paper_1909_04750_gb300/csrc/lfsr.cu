// Bitsliced Fibonacci LFSRs and CRC-8 (Sec. II-B, IV-B, IV-C; Eq. 1, 2;
// Figs. CRC1, CRC2): one thread clocks 32 instances, one 32-bit word per
// register bit, and the register shift is register renaming.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <type_traits>

#include "../../include/bitslice_lfsr.h"
#include "bitslice.cuh"
#include "internal.h"

using namespace mickey;

namespace {

constexpr int kLfsrThreads = 128;
constexpr int kLfsrMaxSparseTaps = 16;  // at most this many taps: lfsr_sparse_kernel
constexpr int kLfsrBlock = 64;                 // clocks per unrolled block of the sparse kernel
constexpr int kLfsrSlots = kLfsrBlock + 64;    // its window: reads reach slot L - 1 + 63
constexpr int kLfsrSparseThreads = 32;  // one warp per block: 1024 blocks even out over the SMs
constexpr int kLfsrBatch = 8;           // clocks per batch of the sparse kernel

struct LfsrMasks {
  uint32_t m[64];  // m[j] = a_{d-1-j} as 0 / ~0 (zero for j >= d)
};

// Instance i's register reversed: y_j = x_{d-1-j}, so that the feedback bit
// enters at y_0 and every other bit moves up one place.  W words hold y in a
// circular buffer: at step u of a W-clock block logical y_j is physical word
// (j - u) mod W and the new bit overwrites the word that falls off, so no
// word moves.  Output t < d is x_t (the seed); output d + c is the feedback
// bit of clock c.
template <int W>
__global__ void __launch_bounds__(kLfsrThreads)
    lfsr_kernel(const uint64_t *seeds, size_t n, int d, LfsrMasks mk, uint64_t n_bits,
                uint32_t *out, uint32_t G) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  // seeds (x) and reversed seeds (y) of the 32 lanes, bitsliced: after
  // transpose32 of rows a[31 - l] = lane l's value, a[c] holds bit 31 - c
  uint32_t xlo[32], xhi[32], y[64];
  {
    uint32_t ylo[32], yhi[32];
#pragma unroll
    for (int l = 0; l < 32; ++l) {
      const uint64_t i = uint64_t(g) * 32 + l;
      const uint64_t v = i < n ? seeds[i] : 0ull;
      const uint64_t rv = __brevll(v) >> (64 - d);
      xlo[31 - l] = uint32_t(v);
      xhi[31 - l] = uint32_t(v >> 32);
      ylo[31 - l] = uint32_t(rv);
      yhi[31 - l] = uint32_t(rv >> 32);
    }
    transpose32(xlo);
    transpose32(xhi);
    transpose32(ylo);
    transpose32(yhi);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      y[j] = ylo[31 - j];
      y[32 + j] = yhi[31 - j];
    }
  }
  const uint64_t head = n_bits < uint64_t(d) ? n_bits : uint64_t(d);
#pragma unroll
  for (int t = 0; t < 64; ++t)
    if (t < int(head)) out[uint64_t(t) * G + g] = t < 32 ? xlo[31 - t] : xhi[63 - t];
  const uint64_t clocks = n_bits - head;
  uint32_t *o = out + uint64_t(d) * G + g;
  // blocks of W clocks whose chains run unguarded, so that the compiler may
  // overlap the XOR chains of neighbouring clocks (only the newest term of a
  // chain depends on the clock before); only the stores past the last
  // requested clock are skipped, the extra clocks' words are discarded
  const uint64_t blocks = (clocks + W - 1) / W;
#pragma unroll 1
  for (uint64_t b = 0; b < blocks; ++b) {
    const uint64_t lim = clocks - b * W;  // >= 1
#pragma unroll
    for (int u = 0; u < W; ++u) {
      uint32_t f = y[(W - u) % W] & mk.m[0];
#pragma unroll
      for (int j = 1; j < W; ++j) f = lop3<0x78>(f, y[(j - u + W) % W], mk.m[j]);
      y[(2 * W - 1 - u) % W] = f;
      if (uint64_t(u) < lim) o[uint64_t(u) * G] = f;
    }
    o += uint64_t(W) * G;
  }
}

// Sparse taps: the recurrence s_{t+d} = XOR over the k taps j of s_{t+j}
// costs k - 1 XORs per clock, not the d masked terms of the kernel above.
// The tap positions are run-time values, and registers cannot be indexed at
// run time, so each thread keeps its words in its own column of shared
// memory: a window of L + 64 slots.  Clocks run in blocks of L = 64 (fully
// unrolled, so every slot offset is an immediate): at the start of a block
// slot s holds x_{c0+s} for s < d; clock u reads slots u + j and writes the
// new word x_{c0+u+d} to slot u + d and, once u + d >= L, also to slot
// u + d - L, where the next block reads it.  That second write lands on a
// slot no later clock of the block reads (reads at clock u' >= u start at
// slot u'), so the window never needs copying; it costs d / L extra stores
// per clock.  Per clock and warp: k shared loads, 1 + d / L shared stores
// and one global store, whose issue bounds the kernel.
struct LfsrTaps {
  uint32_t off[kLfsrMaxSparseTaps];  // tap positions j (a_j = 1), ascending
};

template <int K, int TB>
__device__ __forceinline__ uint32_t lfsr_sparse_clock(const uint32_t *const (&rd)[K], int u) {
  uint32_t f = rd[0][u * TB];
#pragma unroll
  for (int i = 1; i < K; ++i) f ^= rd[i][u * TB];
  return f;
}

// B clocks per batch: the reads of a batch's clocks are all issued before
// any of its writes, so their shared-memory latencies overlap.  Valid when
// no read of a batch needs a word the same batch writes: the newest word a
// clock reads is x_{c+j_max}, written d - j_max clocks earlier, so B <=
// d - j_max.  B = 1 serves every tap set.
template <int K, int TB, int B>
__global__ void __launch_bounds__(TB)
    lfsr_sparse_kernel(const uint64_t *seeds, size_t n, int d, LfsrTaps tp, uint64_t n_bits,
                       uint32_t *out, uint32_t G) {
  constexpr int L = kLfsrBlock;
  extern __shared__ uint32_t lfsr_win[];  // kLfsrSlots x TB words
  const uint32_t g = blockIdx.x * TB + threadIdx.x;
  if (g >= G) return;  // threads use only their own column: no block-wide sync
  uint32_t xlo[32], xhi[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) {
    const uint64_t i = uint64_t(g) * 32 + l;
    const uint64_t v = i < n ? seeds[i] : 0ull;
    xlo[31 - l] = uint32_t(v);
    xhi[31 - l] = uint32_t(v >> 32);
  }
  transpose32(xlo);  // now xlo[31 - t] = word of bit t (t < 32), xhi[63 - t] (t >= 32)
  transpose32(xhi);
  uint32_t *col = lfsr_win + threadIdx.x;
  const uint64_t head = n_bits < uint64_t(d) ? n_bits : uint64_t(d);
#pragma unroll
  for (int t = 0; t < 64; ++t) {
    const uint32_t x = t < 32 ? xlo[31 - t] : xhi[63 - t];
    if (t < d) col[t * TB] = x;
    if (t < int(head)) out[uint64_t(t) * G + g] = x;
  }
  const uint64_t clocks = n_bits - head;
  const uint32_t *rd[K];
#pragma unroll
  for (int i = 0; i < K; ++i) rd[i] = col + tp.off[i] * TB;
  uint32_t *wr = col + d * TB;
  uint32_t *o = out + uint64_t(d) * G + g;
  const uint64_t full = clocks / L;
#pragma unroll 1
  for (uint64_t b = 0; b < full; ++b) {
#pragma unroll
    for (int u0 = 0; u0 < L; u0 += B) {
      uint32_t f[B];
#pragma unroll
      for (int v = 0; v < B; ++v) f[v] = lfsr_sparse_clock<K, TB>(rd, u0 + v);
#pragma unroll
      for (int v = 0; v < B; ++v) {
        const int u = u0 + v;
        wr[u * TB] = f[v];
        if (u + d >= L) wr[(u - L) * TB] = f[v];
        o[uint64_t(u) * G] = f[v];
      }
    }
    o += uint64_t(L) * G;
  }
#pragma unroll 1
  for (int u = 0; u < int(clocks - full * L); ++u) {
    const uint32_t f = lfsr_sparse_clock<K, TB>(rd, u);
    wr[u * TB] = f;
    if (u + d >= L) wr[(u - L) * TB] = f;
    o[uint64_t(u) * G] = f;
  }
}

// CRC-8 of 32 messages per thread (group g = messages 32g .. 32g+31),
// general form (any length and alignment): per pass the thread loads 16
// bytes of each of its 32 messages into registers, transposes each 32 x 32
// bit block (one word per message -> one word per message bit, lane l =
// message l) and clocks the bitsliced register once per bit, bytes in
// order and each byte's most significant bit first.  Each pass uses half of
// a 32-byte sector and leaves the other half to the next pass, which at
// full size mostly finds it evicted from L2: the aligned form below is the
// fast path.
constexpr int kCrcThreads = 64;
constexpr int kCrcChunk = 16;

// The 32 x 32 bit transpose of transpose32 (same result) in fewer ops:
// the 16- and 8-bit block swaps are byte moves, one PRMT per word; the 4-,
// 2- and 1-bit swaps are one shift and one bit-select LOP3 per word.
__device__ __forceinline__ void transpose32_prmt(uint32_t (&a)[32]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint32_t x = a[k], y = a[k + 16];
    a[k] = __byte_perm(x, y, 0x3276);
    a[k + 16] = __byte_perm(x, y, 0x1054);
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k & 8) continue;
    const uint32_t x = a[k], y = a[k + 8];
    a[k] = __byte_perm(x, y, 0x3715);
    a[k + 8] = __byte_perm(x, y, 0x2604);
  }
  auto stage = [&](auto jc, uint32_t m) {
    constexpr int j = decltype(jc)::value;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      if (k & j) continue;
      const uint32_t x = a[k], y = a[k + j];
      a[k] = lop3<0xD8>(x, y >> j, m);               // (x & ~m) | ((y >> j) & m)
      a[k + j] = lop3<0xD8>(y, x << j, m << j);
    }
  };
  stage(std::integral_constant<int, 4>{}, 0x0F0F0F0Fu);
  stage(std::integral_constant<int, 2>{}, 0x33333333u);
  stage(std::integral_constant<int, 1>{}, 0x55555555u);
}

// Message m0 + l's CRC: bit k from s[k], lane l; then the final XOR.
__device__ __forceinline__ void store_crcs(const uint32_t (&s)[8], size_t m0, size_t n,
                                           uint32_t xorout, uint8_t *crc) {
#pragma unroll 1
  for (int l = 0; l < 32; ++l) {
    if (m0 + l >= n) break;
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r |= ((s[k] >> l) & 1u) << k;
    crc[m0 + l] = uint8_t(r ^ xorout);
  }
}

__device__ __forceinline__ uint4 load_chunk(const uint8_t *src, size_t left, bool vec) {
  if (vec && left >= 16) return *reinterpret_cast<const uint4 *>(src);
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int k = 0; k < 16; ++k)
    if (size_t(k) < left) w[k >> 2] |= uint32_t(src[k]) << (8 * (k & 3));
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void __launch_bounds__(kCrcThreads)
    crc8_regs_kernel(const uint8_t *data, size_t n, size_t len, uint32_t poly, uint32_t init,
                     uint32_t xorout, uint8_t *crc, bool vec, size_t G) {
  uint32_t pm[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) pm[k] = (poly >> k) & 1u ? ~0u : 0u;
#pragma unroll 1
  for (size_t g = blockIdx.x * size_t(kCrcThreads) + threadIdx.x; g < G;
       g += size_t(gridDim.x) * kCrcThreads) {
    const size_t m0 = g * 32;
    uint32_t s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = (init >> k) & 1u ? ~0u : 0u;
#pragma unroll 1
    for (size_t off = 0; off < len; off += kCrcChunk) {
      const size_t left = len - off;
      uint4 v[32];
#pragma unroll
      for (int l = 0; l < 32; ++l)
        v[l] = m0 + l < n ? load_chunk(data + (m0 + l) * len + off, left, vec)
                          : make_uint4(0u, 0u, 0u, 0u);
      const int cb = left < size_t(kCrcChunk) ? int(left) : kCrcChunk;   // uniform
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if (4 * w < cb) {
          uint32_t a[32];
#pragma unroll
          for (int l = 0; l < 32; ++l)
            a[31 - l] = w == 0 ? v[l].x : w == 1 ? v[l].y : w == 2 ? v[l].z : v[l].w;
          transpose32_prmt(a);   // a[c]: bit 31 - c of the word, lane l = message l
          const int nbytes = cb - 4 * w < 4 ? cb - 4 * w : 4;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (b < nbytes) {
#pragma unroll
              for (int i = 0; i < 8; ++i) {   // byte b, most significant bit first
                const uint32_t f = s[7] ^ a[24 - 8 * b + i];
#pragma unroll
                for (int k = 7; k > 0; --k) s[k] = lop3<0x78>(s[k - 1], f, pm[k]);
                s[0] = f & pm[0];
              }
            }
          }
        }
      }
    }
    store_crcs(s, m0, n, xorout, crc);
  }
}

// Aligned form (16-byte aligned messages, len % 16 == 0): a block of
// kCrcGroups threads owns kCrcGroups * 32 messages; per pass cp.async copies
// 32 bytes (one whole sector) of each straight into shared memory, about 64
// asynchronous 16-byte copies per thread in flight and no registers held.
// The 16-byte units of group t are XOR-swizzled by t mod 8 within their
// 128-byte row, so that the 16-byte reads of 8 consecutive threads (one
// shared-memory phase) fall on 8 different bank groups.
constexpr int kCrcGroups = 64;
constexpr int kCrcPass = 32;                                   // bytes per message per pass
constexpr size_t kCrcTileBytes = size_t(kCrcGroups) * 32 * kCrcPass;

__device__ __forceinline__ uint32_t crc_unit(uint32_t m, uint32_t c) {
  return (2u * m + c) ^ ((m >> 5) & 7u);
}

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc, uint32_t bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(bytes)
               : "memory");
}

__global__ void __launch_bounds__(kCrcGroups)
    crc8_async_kernel(const uint8_t *data, size_t n, size_t len, uint32_t poly, uint32_t init,
                      uint32_t xorout, uint8_t *crc, size_t n_tiles) {
  extern __shared__ uint4 tile[];
  const uint32_t t = threadIdx.x;
  uint32_t pm[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) pm[k] = (poly >> k) & 1u ? ~0u : 0u;
#pragma unroll 1
  for (size_t blk = blockIdx.x; blk < n_tiles; blk += gridDim.x) {
    const size_t msg0 = blk * kCrcGroups * 32;
    uint32_t s[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k] = (init >> k) & 1u ? ~0u : 0u;
#pragma unroll 1
    for (size_t off = 0; off < len; off += kCrcPass) {
      __syncthreads();   // the previous pass has read the tile
#pragma unroll 8
      for (uint32_t p = t; p < kCrcGroups * 32 * 2; p += kCrcGroups) {
        const uint32_t m = p >> 1, c = p & 1u;
        const size_t msg = msg0 + m, b0 = off + 16 * c;
        const bool in = msg < n && b0 < len;                   // else zero-filled
        cp_async16(tile + crc_unit(m, c), in ? data + msg * len + b0 : data, in ? 16u : 0u);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      const int cb = len - off < size_t(kCrcPass) ? int(len - off) : kCrcPass;   // uniform
#pragma unroll 1
      for (uint32_t c = 0; c < 2; ++c) {
        if (16 * int(c) >= cb) break;
        uint4 v[32];
#pragma unroll
        for (int l = 0; l < 32; ++l) v[l] = tile[crc_unit(32 * t + l, c)];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          uint32_t a[32];
#pragma unroll
          for (int l = 0; l < 32; ++l)
            a[31 - l] = w == 0 ? v[l].x : w == 1 ? v[l].y : w == 2 ? v[l].z : v[l].w;
          transpose32_prmt(a);
#pragma unroll
          for (int b = 0; b < 4; ++b) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const uint32_t f = s[7] ^ a[24 - 8 * b + i];
#pragma unroll
              for (int k = 7; k > 0; --k) s[k] = lop3<0x78>(s[k - 1], f, pm[k]);
              s[0] = f & pm[0];
            }
          }
        }
      }
    }
    store_crcs(s, msg0 + size_t(t) * 32, n, xorout, crc);
  }
}

// Fully coalesced form (16-byte aligned messages, len % 512 == 0): one warp
// per group of 32 messages, lane j taking bytes [16j, 16j + 16) of each
// 512-byte chunk, so one load instruction reads 512 contiguous bytes of one
// message.  CRC is linear over GF(2): a register R run over B bits of data D
// ends at R x^B + CRC0(D) mod P (CRC0: from a zero register).  Lane j keeps
// an accumulator A_j = A_j x^4096 + CRC0(its piece of the chunk), lane 31's
// starting at the preset register; after the last chunk the message's
// register is the sum of A_j x^(128 (31 - j)), which a 5-level shuffle tree
// forms (level k multiplies the left half by x^(128 * 2^k)).  Multiplying by
// a fixed polynomial mod P is an 8 x 8 bit matrix; in bitsliced form each
// output word is the XOR of the input words its row selects.
//
// POLY != 0: the polynomial is a compile-time constant, so the rows are too:
// a product is a fixed XOR network, and a message byte goes in at once as
// (c + B) x^8 mod P (8 XORs and that network; 22 logic ops a byte for 0x1D
// against 32 for its eight bit steps).  POLY == 0: any polynomial, bit by
// bit with run-time masks (9 ops a bit), products as 64 masked LOP3 with the
// rows read from the constant bank.
struct CrcJoin {
  uint32_t m[6][8][8];   // level k, output bit o, input bit i: ~0 if bit o of x^i X_k mod P
};
constexpr int kCrcWarpBlock = 128;

__device__ __forceinline__ void gf2_mul_add(uint32_t (&y)[8], const uint32_t (&x)[8],
                                            const uint32_t (&m)[8][8]) {
#pragma unroll
  for (int o = 0; o < 8; ++o)
#pragma unroll
    for (int i = 0; i < 8; ++i) y[o] = lop3<0x78>(y[o], x[i], m[o][i]);
}

// One message bit x (bitsliced) into register c, most significant bit first.
template <uint32_t POLY>
__device__ __forceinline__ void crc_bit(uint32_t (&c)[8], uint32_t x, const uint32_t (&pm)[8]) {
  const uint32_t f = c[7] ^ x;
  if constexpr (POLY == 0) {
#pragma unroll
    for (int k = 7; k > 0; --k) c[k] = lop3<0x78>(c[k - 1], f, pm[k]);
    c[0] = f & pm[0];
  } else {
    static_for<0, 7>([&](auto kc) {
      constexpr int k = 7 - decltype(kc)::value;          // 7 .. 1
      if constexpr ((POLY >> k) & 1u) c[k] = c[k - 1] ^ f;
      else c[k] = c[k - 1];
    });
    c[0] = (POLY & 1u) ? f : 0u;
  }
}

// Compile-time GF(2)[x] / P arithmetic for the polynomials with their own
// kernel (P = x^8 + POLY): x^e mod P, and the row masks of multiplication
// by x^e (bit j of row o: bit o of x^(j+e) mod P).
__host__ __device__ constexpr uint32_t gf2_xpow_c(uint32_t e, uint32_t P) {
  uint32_t r = 1u, b = 2u;  // r = 1, b = x
  auto mulmod = [](uint32_t u, uint32_t v, uint32_t q) {
    uint32_t t = 0;
    for (int k = 0; k < 8; ++k)
      if ((v >> k) & 1u) t ^= u << k;
    for (int k = 15; k >= 8; --k)
      if ((t >> k) & 1u) t ^= q << (k - 8);
    return t;
  };
  for (; e; e >>= 1) {
    if (e & 1u) r = mulmod(r, b, P);
    b = mulmod(b, b, P);
  }
  return r;
}
template <uint32_t POLY>
__host__ __device__ constexpr uint32_t mulx_row(uint32_t e, int o) {
  uint32_t row = 0;
  for (int j = 0; j < 8; ++j)
    if ((gf2_xpow_c(e + uint32_t(j), 0x100u | POLY) >> o) & 1u) row |= 1u << j;
  return row;
}

// y += x * x^E mod P on bitsliced registers (word k = coefficient of x^k of
// 32 lanes): each output word is the XOR of the input words its row selects.
template <uint32_t POLY, uint32_t E>
__device__ __forceinline__ void mulx_add(uint32_t (&y)[8], const uint32_t (&x)[8]) {
  static_for<0, 8>([&](auto oc) {
    constexpr int o = decltype(oc)::value;
    constexpr uint32_t row = mulx_row<POLY>(E, o);
    static_for<0, 8>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      if constexpr ((row >> j) & 1u) y[o] ^= x[j];
    });
  });
}

// One message byte into register c (the eight bit steps of crc_bit at
// once): after eight steps an MSB-first CRC register is (c + B) x^8 mod P,
// B the byte as a polynomial.  m[j] = bit j of the byte for the 32 lanes.
template <uint32_t POLY>
__device__ __forceinline__ void crc_byte(uint32_t (&c)[8], const uint32_t (&m)[8]) {
  uint32_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = c[j] ^ m[j];
    y[j] = 0u;
  }
  mulx_add<POLY, 8>(y, x);
#pragma unroll
  for (int j = 0; j < 8; ++j) c[j] = y[j];
}

template <uint32_t POLY>
__global__ void __launch_bounds__(kCrcWarpBlock)
    crc8_warp_kernel(const uint8_t *data, size_t n, size_t len, uint32_t poly, uint32_t init,
                     uint32_t xorout, uint8_t *crc, CrcJoin cj, size_t G) {
  constexpr uint32_t F = 0xffffffffu;
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t pm[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) pm[k] = (poly >> k) & 1u ? ~0u : 0u;
  const size_t warps = size_t(gridDim.x) * (kCrcWarpBlock / 32);
#pragma unroll 1
  for (size_t g = size_t(blockIdx.x) * (kCrcWarpBlock / 32) + (threadIdx.x >> 5); g < G;
       g += warps) {
    const size_t m0 = g * 32;
    uint32_t acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = lane == 31 && ((init >> k) & 1u) ? ~0u : 0u;
#pragma unroll 1
    for (size_t off = 0; off < len; off += 512) {
      uint4 v[32];
#pragma unroll
      for (int l = 0; l < 32; ++l)
        v[l] = m0 + l < n
                   ? *reinterpret_cast<const uint4 *>(data + (m0 + l) * len + off + 16 * lane)
                   : make_uint4(0u, 0u, 0u, 0u);
      uint32_t c[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        uint32_t a[32];
#pragma unroll
        for (int l = 0; l < 32; ++l)
          a[31 - l] = w == 0 ? v[l].x : w == 1 ? v[l].y : w == 2 ? v[l].z : v[l].w;
        transpose32_prmt(a);   // a[q]: bit 31 - q of the word, lane bit l = message l
#pragma unroll
        for (int b = 0; b < 4; ++b) {   // bytes in memory order, most significant bit first
          if constexpr (POLY == 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) crc_bit<POLY>(c, a[24 - 8 * b + i], pm);
          } else {
            uint32_t m[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) m[j] = a[31 - 8 * b - j];
            crc_byte<POLY>(c, m);
          }
        }
      }
      if constexpr (POLY == 0)
        gf2_mul_add(c, acc, cj.m[5]);   // acc x^4096 + CRC0(piece)
      else
        mulx_add<POLY, 4096>(c, acc);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = c[k];
    }
    static_for<0, 5>([&](auto levc) {
      constexpr int lev = decltype(levc)::value;
      uint32_t y[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) y[k] = __shfl_down_sync(F, acc[k], 1u << lev);
      if constexpr (POLY == 0)
        gf2_mul_add(y, acc, cj.m[lev]);
      else
        mulx_add<POLY, (128u << lev)>(y, acc);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] = y[k];
    });
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r |= ((__shfl_sync(F, acc[k], 0) >> lane) & 1u) << k;
    if (m0 + lane < n) crc[m0 + lane] = uint8_t(r ^ xorout);
  }
}

// Polynomials with a compile-time kernel (the CRC-8 variants in common use);
// any other runs the run-time-mask kernel.
template <uint32_t POLY>
void launch_crc_warp(uint32_t grid, cudaStream_t st, const uint8_t *d, size_t n, size_t len,
                     uint32_t poly, uint32_t init, uint32_t xorout, uint8_t *crc,
                     const CrcJoin &cj, size_t G) {
  crc8_warp_kernel<POLY><<<grid, kCrcWarpBlock, 0, st>>>(d, n, len, poly, init, xorout, crc, cj,
                                                         G);
}

// Host: x^e mod P over GF(2) (P with its x^8 term), bit k = coefficient of x^k.
uint32_t gf2_mod(uint32_t a, uint32_t P) {
  for (int b = 31; b >= 8; --b)
    if (a >> b & 1u) a ^= P << (b - 8);
  return a;
}
uint32_t gf2_mulmod(uint32_t a, uint32_t b, uint32_t P) {
  uint32_t r = 0;
  for (int k = 0; k < 8; ++k)
    if (b >> k & 1u) r ^= a << k;
  return gf2_mod(r, P);
}
uint32_t gf2_xpow(uint64_t e, uint32_t P) {
  uint32_t r = 1, a = 2;
  while (e) {
    if (e & 1) r = gf2_mulmod(r, a, P);
    a = gf2_mulmod(a, a, P);
    e >>= 1;
  }
  return r;
}

CrcJoin crc_join_matrices(uint8_t poly) {
  const uint32_t P = 0x100u | poly;
  CrcJoin cj{};
  for (int lev = 0; lev < 6; ++lev) {
    const uint32_t X = gf2_xpow(uint64_t(128) << lev, P);
    for (int i = 0; i < 8; ++i) {
      const uint32_t col = gf2_mulmod(1u << i, X, P);   // x^i * X mod P
      for (int o = 0; o < 8; ++o) cj.m[lev][o][i] = (col >> o) & 1u ? ~0u : 0u;
    }
  }
  return cj;
}

template <int K, int B>
cudaError_t launch_lfsr_sparse_b(const uint64_t *seeds, size_t n, int d, const LfsrTaps &tp,
                                 uint64_t n_bits, uint32_t *out, uint32_t G, cudaStream_t st) {
  constexpr int TB = kLfsrSparseThreads;
  const int smem = kLfsrSlots * TB * 4;
  cudaError_t e = cudaFuncSetAttribute(lfsr_sparse_kernel<K, TB, B>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  lfsr_sparse_kernel<K, TB, B><<<(G + TB - 1) / TB, TB, smem, st>>>(seeds, n, d, tp, n_bits,
                                                                     out, G);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_lfsr_sparse_k(const uint64_t *seeds, size_t n, int d, const LfsrTaps &tp,
                                 uint64_t n_bits, uint32_t *out, uint32_t G, cudaStream_t st) {
  const int j_max = int(tp.off[K - 1]);
  if (d - j_max >= kLfsrBatch && !getenv("MICKEY_LFSR_NOBATCH"))
    return launch_lfsr_sparse_b<K, kLfsrBatch>(seeds, n, d, tp, n_bits, out, G, st);
  return launch_lfsr_sparse_b<K, 1>(seeds, n, d, tp, n_bits, out, G, st);
}

template <int K = 1>
cudaError_t launch_lfsr_sparse(int k, const uint64_t *seeds, size_t n, int d, const LfsrTaps &tp,
                               uint64_t n_bits, uint32_t *out, uint32_t G, cudaStream_t st) {
  if constexpr (K > kLfsrMaxSparseTaps) {
    return cudaErrorInvalidValue;
  } else {
    if (k == K) return launch_lfsr_sparse_k<K>(seeds, n, d, tp, n_bits, out, G, st);
    return launch_lfsr_sparse<K + 1>(k, seeds, n, d, tp, n_bits, out, G, st);
  }
}

template <int W>
cudaError_t launch_lfsr(const uint64_t *seeds, size_t n, int d, const LfsrMasks &mk,
                        uint64_t n_bits, uint32_t *out, uint32_t G, cudaStream_t st) {
  lfsr_kernel<W><<<(G + kLfsrThreads - 1) / kLfsrThreads, kLfsrThreads, 0, st>>>(
      seeds, n, d, mk, n_bits, out, G);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

MICKEY_API int mickey_lfsr_generate(const uint64_t *seeds, size_t n_inst, int degree,
                                    uint64_t taps, uint64_t n_bits, uint32_t *out, int mem,
                                    void *stream) {
  if (!seeds || !out || n_inst == 0 || n_bits == 0)
    return set_error(MICKEY_E_ARG, "NULL pointer or empty request");
  if (degree < 2 || degree > 64) return set_error(MICKEY_E_ARG, "degree must be 2..64");
  if ((degree < 64 && (taps >> degree)) || !(taps & 1u))
    return set_error(MICKEY_E_ARG, "taps must lie below the degree and include a_0");
  if (mem != MICKEY_MEM_HOST && mem != MICKEY_MEM_DEVICE)
    return set_error(MICKEY_E_ARG, "mem must be MICKEY_MEM_HOST or MICKEY_MEM_DEVICE");
  if (n_inst > (size_t(1) << 36)) return set_error(MICKEY_E_ARG, "too many instances");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint32_t G = uint32_t((n_inst + 31) / 32);
  LfsrMasks mk{};
  for (int j = 0; j < degree; ++j) mk.m[j] = (taps >> (degree - 1 - j)) & 1u ? ~0u : 0u;
  const uint64_t *d_seeds = seeds;
  uint64_t *tmp = nullptr;
  if (mem == MICKEY_MEM_HOST) {
    if (cudaMallocAsync(reinterpret_cast<void **>(&tmp), n_inst * 8, st) != cudaSuccess ||
        cudaMemcpyAsync(tmp, seeds, n_inst * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return set_error(MICKEY_E_CUDA, "seed upload");
    d_seeds = tmp;
  }
  int k = 0;
  LfsrTaps tp{};
  for (int j = 0; j < degree; ++j)
    if ((taps >> j) & 1u) {
      if (k < kLfsrMaxSparseTaps) tp.off[k] = uint32_t(j);
      ++k;
    }
  const bool sparse = k <= kLfsrMaxSparseTaps && !getenv("MICKEY_LFSR_DENSE");
  cudaError_t e =
      sparse         ? launch_lfsr_sparse(k, d_seeds, n_inst, degree, tp, n_bits, out, G, st)
      : degree <= 16 ? launch_lfsr<16>(d_seeds, n_inst, degree, mk, n_bits, out, G, st)
      : degree <= 32 ? launch_lfsr<32>(d_seeds, n_inst, degree, mk, n_bits, out, G, st)
                     : launch_lfsr<64>(d_seeds, n_inst, degree, mk, n_bits, out, G, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (e != cudaSuccess) return set_error(MICKEY_E_CUDA, "lfsr kernel launch");
  return set_error(MICKEY_OK, "");
}

MICKEY_API int mickey_crc8(const uint8_t *data, size_t n, size_t len, uint8_t poly,
                           uint8_t init, uint8_t xorout, uint8_t *crc, int mem, void *stream) {
  if (!crc || (!data && len)) return set_error(MICKEY_E_ARG, "NULL pointer");
  if (mem != MICKEY_MEM_HOST && mem != MICKEY_MEM_DEVICE)
    return set_error(MICKEY_E_ARG, "mem must be MICKEY_MEM_HOST or MICKEY_MEM_DEVICE");
  if (n == 0) return set_error(MICKEY_OK, "");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint8_t *d_data = data;
  uint8_t *d_crc = crc, *tmp = nullptr;
  if (mem == MICKEY_MEM_HOST) {
    if (cudaMallocAsync(reinterpret_cast<void **>(&tmp), n * len + n, st) != cudaSuccess)
      return set_error(MICKEY_E_OOM, "crc staging");
    if (len && cudaMemcpyAsync(tmp, data, n * len, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return set_error(MICKEY_E_CUDA, "H2D messages");
    d_data = tmp;
    d_crc = tmp + n * len;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool vec = len % 16 == 0 && reinterpret_cast<uintptr_t>(d_data) % 16 == 0;
  if (vec && len % 512 == 0) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crc8_warp_kernel<0>, kCrcWarpBlock,
                                                  0);
    const size_t G = (n + 31) / 32;
    const size_t blocks = (G + kCrcWarpBlock / 32 - 1) / (kCrcWarpBlock / 32);
    const uint32_t grid = uint32_t(std::min<size_t>(blocks, size_t(sms) * std::max(per_sm, 1)));
    const CrcJoin cj = crc_join_matrices(poly);
    switch (poly) {
      case 0x07: launch_crc_warp<0x07>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      case 0x1D: launch_crc_warp<0x1D>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      case 0x2F: launch_crc_warp<0x2F>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      case 0x31: launch_crc_warp<0x31>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      case 0x9B: launch_crc_warp<0x9B>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      case 0xD5: launch_crc_warp<0xD5>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G); break;
      default: launch_crc_warp<0>(grid, st, d_data, n, len, poly, init, xorout, d_crc, cj, G);
    }
  } else if (vec) {
    if (cudaFuncSetAttribute(crc8_async_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(kCrcTileBytes)) != cudaSuccess)
      return set_error(MICKEY_E_CUDA, "crc kernel shared memory");
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crc8_async_kernel, kCrcGroups,
                                                  kCrcTileBytes);
    const size_t n_tiles = (n + kCrcGroups * 32 - 1) / (kCrcGroups * 32);
    const size_t grid = std::min<size_t>(n_tiles, size_t(sms) * std::max(per_sm, 1));
    crc8_async_kernel<<<uint32_t(grid), kCrcGroups, kCrcTileBytes, st>>>(
        d_data, n, len, poly, init, xorout, d_crc, n_tiles);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crc8_regs_kernel, kCrcThreads, 0);
    const size_t G = (n + 31) / 32;
    const size_t blocks = (G + kCrcThreads - 1) / kCrcThreads;
    const size_t grid = std::min<size_t>(blocks, size_t(sms) * std::max(per_sm, 1));
    crc8_regs_kernel<<<uint32_t(grid), kCrcThreads, 0, st>>>(d_data, n, len, poly, init, xorout,
                                                             d_crc, false, G);
  }
  if (cudaGetLastError() != cudaSuccess) return set_error(MICKEY_E_CUDA, "crc kernel launch");
  if (mem == MICKEY_MEM_HOST) {
    if (cudaMemcpyAsync(crc, d_crc, n, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaFreeAsync(tmp, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
      return set_error(MICKEY_E_CUDA, "D2H crc");
  }
  return set_error(MICKEY_OK, "");
}

}  // extern "C"
