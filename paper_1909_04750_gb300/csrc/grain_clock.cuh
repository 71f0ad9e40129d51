// Bitsliced Grain clock (device code shared by the Grain kernels and the
// clock probe).  See grain.cu for the representation: s[0..79] (LFSR) and
// b[0..79] (NFSR) as 32-lane words, register renaming over an 80-clock
// rotation.
#pragma once

#include <cstdint>

#include "bitslice.cuh"

namespace mickey {
namespace grainc {

constexpr int kG = 80;               // register length
constexpr int kGrainThreads = 64;    // groups per block (bitsliced layout)
constexpr int kRing = 160;           // keystream words per thread in the ring
constexpr int kRingStride = 32;      // each warp's ring is [word][lane]

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x96>(a, b, c);
}
__device__ __forceinline__ uint32_t and3(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x80>(a, b, c);
}
__device__ __forceinline__ uint32_t xand(uint32_t a, uint32_t b, uint32_t c) {
  return lop3<0x78>(a, b, c);   // a ^ (b & c)
}

// The filter h(x0, .., x4) = x1+x4+x0x3+x2x3+x3x4+x0x1x2+x0x2x3+x0x2x4+x1x2x4+x2x3x4
// split by its one NFSR input x4: h = H0 + x4 H1 with H0 = x1 + x3(x0 | x2) +
// x0x1x2 and H1 = 1 + x3 + x2(x0 + x1 + x3), both of LFSR bits only (x0..x3 =
// s3, s25, s46, s64): 5 ops, and z = H0 + (x4 & H1) + the b sum.
__device__ __forceinline__ void grain_h01(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3,
                                          uint32_t &h0, uint32_t &h1) {
  h0 = xor3(x1, lop3<0xE0>(x3, x0, x2), and3(x0, x1, x2));   // 0xE0: a & (b | c)
  h1 = lop3<0x87>(x3, x2, xor3(x0, x1, x3));                  // 0x87: ~(a ^ (b & c))
}

// z from the filter halves and the NFSR's seven linear output taps
// b1+b2+b4+b10+b31+b43+b56 (x4 = b63): 5 ops.
template <int R>
__device__ __forceinline__ uint32_t grain_z(const uint32_t (&b)[kG], uint32_t h0, uint32_t h1) {
#define B(i) b[(R + (i)) % kG]
  const uint32_t t1 = xor3(B(1), B(2), B(4));
  const uint32_t t2 = xor3(B(10), B(31), B(43));
  return xor3(t1, t2, B(56)) ^ xand(h0, B(63), h1);
#undef B
}

// NFSR feedback s0 + g(b), the 23 terms in a tree (at most five dependent
// steps), into slot R; s0 is the LFSR's oldest bit.
template <int R, bool INIT>
__device__ __forceinline__ void grain_nfsr(uint32_t (&b)[kG], uint32_t s0, uint32_t z) {
#define B(i) b[(R + (i)) % kG]
  const uint32_t p1 = B(63) & B(60);
  const uint32_t p2 = B(37) & B(33);
  const uint32_t p3 = B(15) & B(9);
  const uint32_t q = B(60) & B(52);
  const uint32_t r = B(52) & B(45);
  const uint32_t p5 = and3(B(33), B(28), B(21));
  const uint32_t p6 = and3(B(63), B(45), B(28));
  const uint32_t l1 = xor3(B(62), B(60), B(52));
  const uint32_t l2 = xor3(B(45), B(37), B(33));
  const uint32_t l3 = xor3(B(28), B(21), B(14));
  const uint32_t l4 = xor3(B(9), B(0), s0);
  const uint32_t m1 = xor3(l1, l2, l3);                 // the linear terms ...
  const uint32_t m2 = xor3(l4, p1, p2);                 // ... s0, b63b60, b37b33
  const uint32_t m3 = xand(p3, q, B(45));               // b15b9, b60b52b45
  const uint32_t m4 = xand(p5, p6, B(9));               // b33b28b21, b63b45b28b9
  const uint32_t t8 = and3(p1, B(21), B(15));           // b63b60b21b15
  const uint32_t t9 = and3(p1, r, B(37));               // b63b60b52b45b37
  const uint32_t t11 = and3(r, B(37), p5);              // b52b45b37b33b28b21
  const uint32_t n1 = xor3(m1, m2, m3);
  const uint32_t n2 = xand(m4, q, p2);                  // b60b52b37b33
  const uint32_t n3 = xor3(t8, t9, t11);
  const uint32_t n4 = xand(n2, p5, p3);                 // b33b28b21b15b9
  uint32_t nb = xor3(n1, n4, n3);
  if (INIT) nb ^= z;
  B(0) = nb;   // slot R: the oldest bit becomes the newest
#undef B
}

// LFSR feedback s62+s51+s38+s23+s13+s0 (+ z while initialising) into slot R;
// returns the oldest bit s0 it replaces.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t grain_lfsr(uint32_t (&s)[kG], uint32_t z) {
#define S(i) s[(R + (i)) % kG]
  const uint32_t s0 = S(0);
  const uint32_t la = xor3(S(62), S(51), S(38));
  const uint32_t lb = xor3(S(23), S(13), s0);
  S(0) = INIT ? xor3(la, lb, z) : la ^ lb;
  return s0;
#undef S
}

// One clock at rotation R (compile-time): returns z of the current state
// and replaces slot R of both registers by the new bits.  The XOR sums are
// balanced trees, so that the instructions of one clock can issue back to
// back: 36 ops (LFSR 3, NFSR 23, z 10), 37 while initialising.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t grain_clock(uint32_t (&s)[kG], uint32_t (&b)[kG]) {
#define S(i) s[(R + (i)) % kG]
  uint32_t h0, h1;
  grain_h01(S(3), S(25), S(46), S(64), h0, h1);
#undef S
  const uint32_t z = grain_z<R>(b, h0, h1);
  const uint32_t s0 = grain_lfsr<R, INIT>(s, z);
  grain_nfsr<R, INIT>(b, s0, z);
  return z;
}

// 80 clocks (one full rotation); keystream word of clock c to zb[c * kRingStride].
template <bool INIT>
__device__ __forceinline__ void grain_body(uint32_t (&s)[kG], uint32_t (&b)[kG], uint32_t *zb) {
  static_for<0, kG>([&](auto rc) {
    constexpr int R = decltype(rc)::value;
    const uint32_t z = grain_clock<R, INIT>(s, b);
    if constexpr (!INIT) zb[R * kRingStride] = z;
  });
}

// One clock with the registers physically shifted (rotation stays 0): the
// tail of a call, fewer than 80 clocks.
__device__ __forceinline__ uint32_t grain_clock_shift(uint32_t (&s)[kG], uint32_t (&b)[kG]) {
  const uint32_t s0 = s[0], b0 = b[0];
  const uint32_t z = grain_clock<0, false>(s, b);   // writes the new bits to slot 0
  const uint32_t ns = s[0], nb = b[0];
  s[0] = s0;
  b[0] = b0;
  static_for<0, kG - 1>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    s[i] = s[i + 1];
    b[i] = b[i + 1];
  });
  s[kG - 1] = ns;
  b[kG - 1] = nb;
  return z;
}

}  // namespace grainc
}  // namespace mickey
