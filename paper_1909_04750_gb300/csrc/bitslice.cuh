// Bitsliced MICKEY 2.0 clock and bit-matrix transpose (device code).
//
// Representation (Sec. IV-A): r[i] / s[i] is a 32-bit word whose bit l is
// register bit i of lane l, so one thread clocks 32 instances at once with
// full-width logic (Sec. IV-D: 200 words, 32 keystream bits per clock).
//
// The shift of each register is not executed: new word i is computed from
// old words i-1, i, i+1 directly (register renaming, Sec. IV-C), and every
// table constant is a compile-time value, so each register bit costs one
// LOP3, plus one XOR where feedback enters.
#pragma once

#include <cstdint>

#include "tables.cuh"

namespace mickey {

// Feedback contribution to S'_i: FB0_i & fb when CONTROL_BIT_S = 0 and
// FB1_i & fb when it is 1, i.e. one of {0, fb, fb&~cbs, fb&cbs}.
template <int I>
__device__ __forceinline__ uint32_t s_feedback(uint32_t fb, uint32_t f0,
                                               uint32_t f1) {
  if constexpr (fb0(I) && fb1(I))
    return fb;
  else if constexpr (fb0(I))
    return f0;
  else if constexpr (fb1(I))
    return f1;
  else
    return 0u;
}

// d = f(a, b, c) for the truth table LUT (bit 4a + 2b + c of LUT), as one
// three-input logic instruction.  Written out so that every register bit
// of the clock below is exactly the one or two instructions it needs.
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

// Truth table of a ^ ((b ^ C0) & (c ^ C1)) for constant C0, C1 (all-ones or
// zero): the S update of one bit from s_{i-1}, s_i, s_{i+1}.
__host__ __device__ constexpr uint32_t s_lut(bool c0, bool c1) {
  return (0xF0u ^ ((0xCCu ^ (c0 ? 0xFFu : 0u)) & (0xAAu ^ (c1 ? 0xFFu : 0u)))) & 0xFFu;
}

// The values every bit update of a clock reads besides its neighbours:
// CONTROL_BIT_R, the R and S feedback bits, and FB & ~CBS, FB & CBS.
struct KgFeed {
  uint32_t cbr, fbr, fbs, f0, f1;
};

template <bool MIX>
__device__ __forceinline__ KgFeed kg_feed(const uint32_t (&r)[kReg], const uint32_t (&s)[kReg],
                                          uint32_t in) {
  KgFeed f;
  f.cbr = s[34] ^ r[67];
  f.fbr = r[99];
  f.fbs = s[99];
  if constexpr (MIX) {
    f.fbr = lop3<0x96>(f.fbr, in, s[50]);
    f.fbs = f.fbs ^ in;
  }
  f.f0 = lop3<0x90>(f.fbs, s[67], r[33]);   // fbs & ~(s67 ^ r33)
  f.f1 = lop3<0x60>(f.fbs, s[67], r[33]);   // fbs &  (s67 ^ r33)
  return f;
}

// The bit updates of one clock from its feed values (clock_kg below).
template <bool MASK>
__device__ __forceinline__ void clock_kg_from(uint32_t (&r)[kReg], uint32_t (&s)[kReg],
                                              const KgFeed &fd, uint32_t act) {
  const uint32_t cbr = fd.cbr, fbr = fd.fbr, fbs = fd.fbs, f0 = fd.f0, f1 = fd.f1;
  uint32_t nr[kReg], ns[kReg];
  // CLOCK_R: r'_i = r_{i-1} ^ (cbr & r_i) ^ (i in RTAPS ? fb : 0), r_{-1} = 0
  nr[0] = lop3<0x6A>(cbr, r[0], fbr);                  // (cbr & r0) ^ fb
  static_for<1, kReg>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    uint32_t v = lop3<0x78>(r[i - 1], cbr, r[i]);
    if constexpr (rtap(i)) v ^= fbr;
    nr[i] = v;
  });
  // CLOCK_S: s^_i = s_{i-1} ^ ((s_i ^ COMP0_i) & (s_{i+1} ^ COMP1_i)),
  // s^_0 = 0, s^_99 = s_98, then the FB0/FB1 feedback.
  ns[0] = fbs;
  static_for<1, kReg - 1>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    uint32_t v;
    if constexpr (MASK && comp0(i) && comp1(i))
      v = s[i - 1] ^ lop3<0x02>(s[i], s[i + 1], act);  // ~s_i & ~s_{i+1} & act
    else
      v = lop3<s_lut(comp0(i), comp1(i))>(s[i - 1], s[i], s[i + 1]);
    if constexpr (fb0(i) || fb1(i)) v ^= s_feedback<i>(fbs, f0, f1);
    ns[i] = v;
  });
  ns[kReg - 1] = s[kReg - 2] ^ s_feedback<kReg - 1>(fbs, f0, f1);

  static_for<0, kReg>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    r[i] = nr[i];
    s[i] = ns[i];
  });
}

// One bitsliced CLOCK_KG for 32 lanes.
//   MIX   mixing mode (key/IV loading and preclocks): the R input takes
//         in ^ s50, both feedbacks take `in` (bit l = input bit of lane l).
//   MASK  lanes whose bit in `act` is 0 keep their state.  Only used while
//         lanes with shorter IVs have not started their IV clocks: such a
//         lane's state is all zero and its input bits are zero, and a clock
//         of the zero state with zero input changes nothing except the S
//         positions i where COMP0_i = COMP1_i = 1 (s^_i gets c0 & c1 = 1),
//         so AND-ing `act` into the non-linear term of exactly those
//         positions keeps inactive lanes at zero.
// Both registers are clocked from the old state (control bits
// CONTROL_BIT_R = s34 ^ r67, CONTROL_BIT_S = s67 ^ r33).  Instruction
// count: one per bit of R and of S, one more where feedback enters, and
// CBR, FB&~CBS, FB&CBS (CBS folded into the last two).
template <bool MIX, bool MASK>
__device__ __forceinline__ void clock_kg(uint32_t (&r)[kReg],
                                         uint32_t (&s)[kReg], uint32_t in,
                                         uint32_t act) {
  clock_kg_from<MASK>(r, s, kg_feed<MIX>(r, s, in), act);
}

// In-register transpose of a 32 x 32 bit matrix.  Row k is a[k]; column c
// is bit (31 - c).  Afterwards a[c] bit (31 - k) equals the old a[k] bit
// (31 - c).  Five stages swap the off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
  auto stage = [&](auto jc, uint32_t m) {
    constexpr int j = decltype(jc)::value;
    static_for<0, 32>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      if constexpr ((k & j) == 0) {
        const uint32_t t = (a[k] ^ (a[k + j] >> j)) & m;
        a[k] ^= t;
        a[k + j] ^= t << j;
      }
    });
  };
  stage(std::integral_constant<int, 16>{}, 0x0000FFFFu);
  stage(std::integral_constant<int, 8>{}, 0x00FF00FFu);
  stage(std::integral_constant<int, 4>{}, 0x0F0F0F0Fu);
  stage(std::integral_constant<int, 2>{}, 0x33333333u);
  stage(std::integral_constant<int, 1>{}, 0x55555555u);
}

// Block swaps of the two-pass 32x32 transpose used to un-bitslice a tile
// (see the keystream kernels).
template <int J>
__device__ __forceinline__ void swap_bits(uint32_t &lo, uint32_t &hi) {
  // two independent bit-selects, (x & ~m) | (y & m) = truth table 0xD8
  constexpr uint32_t m = J == 4 ? 0x0F0F0F0Fu : J == 2 ? 0x33333333u : 0x55555555u;
  const uint32_t x = lo, y = hi;
  lo = lop3<0xD8>(x, y >> J, m);
  hi = lop3<0xD8>(y, x << J, m << J);
}
// Block swap of size 16: lo keeps its high half and takes hi's high half;
// hi keeps its low half and takes lo's low half.
__device__ __forceinline__ void swap_halves(uint32_t &lo, uint32_t &hi) {
  const uint32_t a = __byte_perm(lo, hi, 0x3276);
  hi = __byte_perm(lo, hi, 0x1054);
  lo = a;
}
// Block swap of size 8 (bytes 1 and 3 of hi into bytes 0 and 2 of lo and
// bytes 0 and 2 of lo into bytes 1 and 3 of hi).  With BSWAP the two results
// come out byte-reversed (the selectors read in the opposite byte order),
// which turns a big-endian word into its memory byte order for free.
template <bool BSWAP>
__device__ __forceinline__ void swap_bytes(uint32_t &lo, uint32_t &hi) {
  const uint32_t a = __byte_perm(lo, hi, BSWAP ? 0x5173 : 0x3715);
  hi = __byte_perm(lo, hi, BSWAP ? 0x4062 : 0x2604);
  lo = a;
}

}  // namespace mickey
