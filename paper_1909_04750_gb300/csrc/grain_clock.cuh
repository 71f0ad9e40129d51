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

// One clock at rotation R (compile-time): returns z of the current state
// and replaces slot R of both registers by the new bits.  The XOR sums are
// balanced trees (at most five dependent steps to the new NFSR bit, four to
// z), so that the instructions of one clock can issue back to back.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t grain_clock(uint32_t (&s)[kG], uint32_t (&b)[kG]) {
#define S(i) s[(R + (i)) % kG]
#define B(i) b[(R + (i)) % kG]
  // output: z = b1+b2+b4+b10+b31+b43+b56 + h(x0..x4),
  // h = A + x2 B, A = x1+x4+x3(x0+x4), B = x3+x4(x1+x3)+x0(x1+x3+x4)
  const uint32_t x0 = S(3), x1 = S(25), x2 = S(46), x3 = S(64), x4 = B(63);
  const uint32_t t1 = xor3(B(1), B(2), B(4));
  const uint32_t t2 = xor3(B(10), B(31), B(43));
  const uint32_t u0 = xor3(x1, x4, B(56));
  const uint32_t t = x0 ^ x4;
  const uint32_t w = x1 ^ x3;
  const uint32_t v = xor3(x1, x3, x4);
  const uint32_t u = xor3(t1, t2, u0);                 // x1 + x4 + (b sum)
  const uint32_t c = xand(x3, x4, w);                  // x3 + x4(x1 + x3)
  const uint32_t a = xand(u, x3, t);                   // A + (b sum)
  const uint32_t bb = xand(c, x0, v);                  // B
  const uint32_t z = xand(a, x2, bb);                  // A + x2 B + (b sum)
  // LFSR: s62+s51+s38+s23+s13+s0 (+ z while initialising)
  const uint32_t la = xor3(S(62), S(51), S(38));
  const uint32_t lb = xor3(S(23), S(13), S(0));
  const uint32_t ns = INIT ? xor3(la, lb, z) : la ^ lb;
  // NFSR: s0 + g(b), the 23 terms in a tree
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
  const uint32_t l4 = xor3(B(9), B(0), S(0));
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
  S(0) = ns;   // slot R: the oldest bit becomes the newest
  B(0) = nb;
#undef S
#undef B
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
