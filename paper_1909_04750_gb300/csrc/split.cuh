// Split clock: one warp clocks one 32-lane group (device code shared by the
// batched and the served kernels).
#pragma once

#include <cstdint>

#include "tables.cuh"

namespace mickey {

// Split path for long groups: one warp clocks one group, so a clock costs
// about 34 logic ops per lane instead of ~390 per thread.  Lane j (< 25) owns
// register bits 4j .. 4j+3 of R and of S (slots 0..3); lanes 25..31 carry
// no bits.  Each clock the warp exchanges neighbour words (r_{4j-1},
// s_{4j-1}, s_{4j+4}) and broadcasts the control and feedback words (s34,
// r67, s67, r33, r99, s99) with shuffles; the table constants become per-lane
// masks.  The keystream word z = r0 ^ s0 (lane 0) is broadcast each clock
// and kept by lane c for clock c; every 32 clocks 32 ballots give each lane
// its instance's 32 bits.

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
  uint32_t tap[4], c0[4], c1[4], en[4], fb0[4], fb1[4];
};

__device__ __forceinline__ void split_lane_masks(uint32_t lane, SplitLane &k) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = int(4 * lane) + q;
    k.tap[q] = bit_mask(kSplitMasks.rtap, i);
    k.c0[q] = bit_mask(kSplitMasks.comp0, i);
    k.c1[q] = bit_mask(kSplitMasks.comp1, i);
    k.fb0[q] = bit_mask(kSplitMasks.fb0, i);
    k.fb1[q] = bit_mask(kSplitMasks.fb1, i);
    // non-linear term of s^_i exists for i = 1..98 only
    k.en[q] = (i >= 1 && i <= 98) ? ~0u : 0u;
  }
}

// One non-mixing CLOCK_KG of the group spread over the warp.
__device__ __forceinline__ void clock_split(uint32_t (&r)[4], uint32_t (&s)[4], const SplitLane &k,
                                            uint32_t lane) {
  constexpr uint32_t F = 0xffffffffu;
  const uint32_t up_ok = lane ? ~0u : 0u;
  const uint32_t r_up = __shfl_up_sync(F, r[3], 1) & up_ok;   // r_{4j-1} (r_{-1} = 0)
  const uint32_t s_up = __shfl_up_sync(F, s[3], 1) & up_ok;   // s_{4j-1}
  const uint32_t s_dn = __shfl_down_sync(F, s[0], 1);         // s_{4j+4}
  const uint32_t cbr = __shfl_sync(F, s[2], 8) ^ __shfl_sync(F, r[3], 16);   // s34 ^ r67
  const uint32_t cbs = __shfl_sync(F, s[3], 16) ^ __shfl_sync(F, r[1], 8);   // s67 ^ r33
  const uint32_t fbr = __shfl_sync(F, r[3], 24);                              // r99
  const uint32_t fbs = __shfl_sync(F, s[3], 24);                              // s99
  const uint32_t f0 = fbs & ~cbs, f1 = fbs & cbs;
  uint32_t nr[4], ns[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const uint32_t rm1 = q ? r[q - 1] : r_up;
    nr[q] = rm1 ^ (cbr & r[q]) ^ (fbr & k.tap[q]);
    const uint32_t sm1 = q ? s[q - 1] : s_up;
    const uint32_t sp1 = q < 3 ? s[q + 1] : s_dn;
    // bits 0 and 99 (no non-linear term) sit in slots 0 and 3 only; the
    // dummy lanes' results never reach a real bit
    const uint32_t a = (q == 0 || q == 3) ? ((s[q] ^ k.c0[q]) & k.en[q]) : (s[q] ^ k.c0[q]);
    const uint32_t nl = a & (sp1 ^ k.c1[q]);
    ns[q] = sm1 ^ nl ^ (f0 & k.fb0[q]) ^ (f1 & k.fb1[q]);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q] = nr[q];
    s[q] = ns[q];
  }
}

// One clock plus keeping z = r0 ^ s0 (lane 0's slot 0) of clock c in lane c.
__device__ __forceinline__ void split_step(uint32_t (&r)[4], uint32_t (&s)[4], const SplitLane &k,
                                           uint32_t lane, int c, uint32_t &zt) {
  const uint32_t z = __shfl_sync(0xffffffffu, r[0] ^ s[0], 0);
  zt = lane == uint32_t(c) ? z : zt;
  clock_split(r, s, k, lane);
}

}  // namespace mickey
