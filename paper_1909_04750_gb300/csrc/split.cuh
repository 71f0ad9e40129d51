// Split clock: one warp clocks one 32-lane group (device code shared by the
// batched and the served kernels).
#pragma once

#include <cstdint>

#include "tables.cuh"

namespace mickey {

// Split path for long groups, where the time per clock of one group (and
// not the throughput of many) bounds the run.  Layout: lane j owns
// R bits 4j .. 4j+3 (slot q = bit 4j+q, lanes 0..24) and S bits 100-4j ..
// 97-4j in reverse (slot q = bit 100-4j-q, lanes 0..25); the slots outside
// 0..99 hold zeros that stay zero, except S bit 100 (lane 0, slot 0), which
// only ever feeds the disabled non-linear term of bit 99.  With S reversed,
// s34 sits beside r67 (lane 16) and s67 beside r33 (lane 8), so each control
// bit is XORed in its lane and broadcast once, and all six control and
// feedback bits (r33, r67, r99, s34, s67, s99) have both neighbours in their
// own lane: the neighbour shuffles stay off the clock-to-clock chain.  One
// clock per lane:
//   * 7 shuffles: r_{4j-1}, the two S neighbour words, CBR, CBS, r99, s99;
//   * R: r'_i = r_{i-1} ^ (CBR & r_i) ^ (fb_R & [i in RTAPS]), 2 LOP3 a slot;
//   * S: the table constants of bit i are lane-dependent, so the terms that
//     XOR or AND a word with one of them, s_i ^ COMP0_i (zero outside
//     i = 1..98), s_{i+1} ^ COMP1_i and FB0_i ^ (CBS & (FB0_i ^ FB1_i)), are
//     each x * m + a with m in {0, 1, -1} and a in {0, -1} (IMAD, on the FMA
//     pipe beside the logic pipe); two LOP3 combine them.
// Lane 0 stores r0 and lane 25 stores s0 (before the clock) to the warp's
// shared memory; after 32 clocks their XOR, one word per clock, goes
// through a 5-stage xor-shuffle butterfly that transposes the 32 x 32 bit
// tile, so lane l holds its instance's 32 bits.

// clocks per iteration of the split path's tile loop (the whole tile)
constexpr int kSplitUnroll = 32;
// S bit held by slot q of lane j (R bit: 4j + q)
__host__ __device__ constexpr int split_s_bit(int j, int q) { return 100 - 4 * j - q; }

struct SplitMasks {
  uint32_t rtap[4], comp0[4], comp1[4], fb0[4], fb1[4];
};
constexpr SplitMasks make_split_masks() {
  SplitMasks m{};
  for (int i = 0; i < kReg; ++i) {
    const uint32_t b = 1u << (i % 32);
    if (rtap(i)) m.rtap[i / 32] |= b;
    if (comp0(i)) m.comp0[i / 32] |= b;
    if (comp1(i)) m.comp1[i / 32] |= b;
    if (fb0(i)) m.fb0[i / 32] |= b;
    if (fb1(i)) m.fb1[i / 32] |= b;
  }
  return m;
}
static __constant__ SplitMasks kSplitMasks = make_split_masks();

__device__ __forceinline__ uint32_t bit_mask(const uint32_t (&w)[4], int i) {
  return (i < kReg && ((w[i >> 5] >> (i & 31)) & 1u)) ? ~0u : 0u;
}

struct SplitLane {
  uint32_t src_up_r, src_up_s, src_dn_s;          // shuffle sources of the neighbour words
  uint32_t zm;                                    // ~0 in lane 25 (z from s0), else 0
  uint32_t tap[4];                                // RTAPS as 0 / ~0
  uint32_t c0m[4], c0a[4], c1m[4], c1a[4], fbm[4], fba[4];   // IMAD coefficients
  uint32_t tmask[5], tshift[5];                   // butterfly transpose stages
};

__device__ __forceinline__ void split_lane_init(uint32_t lane, SplitLane &k) {
  // lane 0 reads lane 31 (zero); the zero lanes read themselves, so nothing
  // ever reaches them
  k.src_up_r = lane == 0 ? 31u : (lane <= 24 ? lane - 1 : lane);
  k.src_up_s = lane == 0 ? 31u : (lane <= 25 ? lane - 1 : lane);
  k.src_dn_s = lane <= 25 ? lane + 1 : lane;
  k.zm = lane == 25 ? ~0u : 0u;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    k.tap[q] = bit_mask(kSplitMasks.rtap, int(4 * lane) + q);
    const int i = split_s_bit(int(lane), q);
    const uint32_t c0 = bit_mask(kSplitMasks.comp0, i), c1 = bit_mask(kSplitMasks.comp1, i);
    const uint32_t f0 = bit_mask(kSplitMasks.fb0, i), f1 = bit_mask(kSplitMasks.fb1, i);
    const bool en = i >= 1 && i <= 98;          // the non-linear term exists for 1..98
    k.c0m[q] = en ? (c0 ? ~0u : 1u) : 0u;       // (s ^ c0) & en
    k.c0a[q] = en ? c0 : 0u;
    k.c1m[q] = c1 ? ~0u : 1u;                   // x ^ c1
    k.c1a[q] = c1;
    k.fbm[q] = (f0 ^ f1) ? (f0 ? ~0u : 1u) : 0u;   // f0 ^ (cbs & (f0 ^ f1))
    k.fba[q] = f0;
  }
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const uint32_t j = 16u >> st;
    constexpr uint32_t kLow[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
    const bool top = (lane & j) == 0;
    k.tmask[st] = top ? kLow[st] : ~kLow[st];
    k.tshift[st] = top ? j : 32u - j;
  }
}

// d = a ^ (b & c) as one three-input logic op (truth table 0xf0 ^ (0xcc &
// 0xaa) = 0x78), so that each slot's update is exactly two of them.
__device__ __forceinline__ uint32_t xor_and(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x78;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// One non-mixing CLOCK_KG of the group spread over the warp.
__device__ __forceinline__ void clock_split(uint32_t (&r)[4], uint32_t (&s)[4],
                                            const SplitLane &k) {
  constexpr uint32_t F = 0xffffffffu;
  const uint32_t cbr = __shfl_sync(F, s[2] ^ r[3], 16);   // s34 ^ r67
  const uint32_t cbs = __shfl_sync(F, s[1] ^ r[1], 8);    // s67 ^ r33
  const uint32_t fbr = __shfl_sync(F, r[3], 24);          // r99
  const uint32_t fbs = __shfl_sync(F, s[1], 0);           // s99
  const uint32_t r_up = __shfl_sync(F, r[3], k.src_up_r); // r_{4j-1}
  const uint32_t s_up = __shfl_sync(F, s[3], k.src_up_s); // s_{i+1} of slot 0
  const uint32_t s_dn = __shfl_sync(F, s[0], k.src_dn_s); // s_{i-1} of slot 3
  uint32_t nr[4], ns[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t rm1 = q ? r[q - 1] : r_up;
    nr[q] = xor_and(xor_and(rm1, cbr, r[q]), fbr, k.tap[q]);
    const uint32_t sm1 = q < 3 ? s[q + 1] : s_dn;
    const uint32_t sp1 = q ? s[q - 1] : s_up;
    const uint32_t y = s[q] * k.c0m[q] + k.c0a[q];
    const uint32_t z = sp1 * k.c1m[q] + k.c1a[q];
    const uint32_t sel = cbs * k.fbm[q] + k.fba[q];
    ns[q] = xor_and(xor_and(sm1, y, z), fbs, sel);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q] = nr[q];
    s[q] = ns[q];
  }
}

// n <= 32 clocks of the group, then the transpose: returns lane's
// instance's bits, clock c in bit c (bits >= n zero).  zbuf0 / zbuf1: 32
// words each of shared memory owned by the warp (r0 and s0 of each clock).
template <int SU>
__device__ __forceinline__ uint32_t split_tile(uint32_t (&r)[4], uint32_t (&s)[4],
                                               const SplitLane &k, uint32_t lane,
                                               uint32_t *zbuf0, uint32_t *zbuf1, int n) {
  const bool lead = lane == 0 || lane == 25;
  uint32_t *zb = lane == 25 ? zbuf1 : zbuf0;
  if (n == 32) {
#pragma unroll 1
    for (int c = 0; c < 32; c += SU) {
#pragma unroll
      for (int u = 0; u < SU; ++u) {
        if (lead) zb[c + u] = xor_and(r[0], s[0], k.zm);   // r0 (lane 0), s0 (lane 25)
        clock_split(r, s, k);
      }
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < n; ++c) {
      if (lead) zb[c] = xor_and(r[0], s[0], k.zm);
      clock_split(r, s, k);
    }
  }
  __syncwarp();
  uint32_t x = lane < uint32_t(n) ? zbuf0[lane] ^ zbuf1[lane] : 0u;
  __syncwarp();
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, 16 >> st);
    x = (x & k.tmask[st]) | (__funnelshift_l(y, y, k.tshift[st]) & ~k.tmask[st]);
  }
  return x;
}

}  // namespace mickey
