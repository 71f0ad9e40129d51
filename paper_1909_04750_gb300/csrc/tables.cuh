// MICKEY 2.0 constant tables as compile-time index sets.
//
// Each list holds the register positions i (0..99) where the table entry
// is 1, transcribed from the cipher specification's tables (the cipher the
// paper bitslices, Sec. II-C-1 / IV-D).  In the kernels every entry is a
// compile-time constant, so the per-bit logic of CLOCK_R / CLOCK_S folds into
// one 3-input LOP3 per bit plus one XOR per feedback position.
#pragma once

#include <cstdint>
#include <type_traits>

namespace mickey {

constexpr int kReg = 100;

// R: feedback tap positions.
constexpr int kRTaps[] = {0,  1,  3,  4,  5,  6,  9,  12, 13, 16, 19, 20, 21,
                          22, 25, 28, 37, 38, 41, 42, 45, 46, 50, 52, 54, 56,
                          58, 60, 61, 63, 64, 65, 66, 67, 71, 72, 79, 80, 81,
                          82, 87, 88, 89, 90, 91, 92, 94, 95, 96, 97};
// S: positions with COMP0_i = 1 (defined for i = 1..98).
constexpr int kComp0[] = {4,  5,  9,  11, 12, 13, 14, 16, 19, 21, 23, 25, 27,
                          29, 30, 32, 35, 43, 45, 47, 49, 54, 56, 59, 60, 61,
                          62, 65, 67, 69, 70, 71, 72, 73, 74, 75, 76, 77, 79,
                          81, 82, 83, 84, 85, 86, 88, 90, 97, 98};
// S: positions with COMP1_i = 1 (defined for i = 1..98).
constexpr int kComp1[] = {1,  3,  4,  7,  9,  10, 11, 12, 15, 17, 21, 22, 24,
                          26, 27, 28, 30, 31, 32, 33, 37, 38, 40, 42, 43, 44,
                          49, 53, 55, 56, 57, 61, 62, 63, 64, 65, 66, 68, 70,
                          71, 72, 74, 75, 76, 77, 81, 86, 87, 88, 92, 95, 96};
// S: positions with FB0_i = 1 (feedback when CONTROL_BIT_S = 0).
constexpr int kFb0[] = {0,  1,  2,  3,  5,  7,  8,  9,  10, 11, 12, 13, 14, 17,
                        19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 31, 32, 39, 40,
                        41, 44, 47, 49, 51, 54, 56, 57, 58, 59, 61, 63, 65, 75,
                        76, 78, 82, 83, 85, 86, 87, 90, 91, 92, 95, 96};
// S: positions with FB1_i = 1 (feedback when CONTROL_BIT_S = 1).
constexpr int kFb1[] = {0,  1,  2,  4,  5,  6,  11, 12, 13, 15, 18, 19,
                        23, 26, 27, 30, 32, 33, 37, 38, 44, 45, 47, 48,
                        52, 56, 59, 62, 64, 65, 67, 69, 72, 74, 78, 79,
                        80, 81, 83, 84, 85, 86, 87, 94, 99};

template <int N>
__host__ __device__ constexpr bool contains(const int (&a)[N], int i) {
  for (int k = 0; k < N; ++k)
    if (a[k] == i) return true;
  return false;
}
__host__ __device__ constexpr bool rtap(int i) { return contains(kRTaps, i); }
__host__ __device__ constexpr bool comp0(int i) { return contains(kComp0, i); }
__host__ __device__ constexpr bool comp1(int i) { return contains(kComp1, i); }
__host__ __device__ constexpr bool fb0(int i) { return contains(kFb0, i); }
__host__ __device__ constexpr bool fb1(int i) { return contains(kFb1, i); }

static_assert(sizeof(kRTaps) / sizeof(int) == 50, "RTAPS has 50 taps");
static_assert(rtap(0), "R bit 0 is a tap; the clock relies on it");
static_assert(fb0(0) && fb1(0), "S'_0 = feedback in both control cases");

// Number of S positions 1..98 that receive feedback under either control.
__host__ __device__ constexpr int s_feedback_positions() {
  int c = 0;
  for (int i = 1; i <= 98; ++i) c += (fb0(i) || fb1(i)) ? 1 : 0;
  return c;
}

// Algorithmic 32-bit logic ops of one bitsliced CLOCK_KG per 32 lanes, with
// constants folded into 3-input LOP3 (the counting used for the roofline):
//   CONTROL_BIT_R                      1
//   R'_0 = (cbr & r0) ^ fb             1
//   R'_i, i = 1..99: one LOP3, +1 XOR at a tap
//   f0 = fb_s & ~cbs, f1 = fb_s & cbs  2   (cbs folded into both)
//   S'_0 = fb_s                        0   (renaming)
//   S'_i, i = 1..98: one LOP3, +1 XOR at a feedback position
//   S'_99 = s98 ^ (fb term)            1
//   keystream: z = r0 ^ s0             1
//   mixing: in_r = in ^ s50, fb_r ^= in_r, fb_s ^= in   3
__host__ __device__ constexpr int ops_per_clock(bool mixing) {
  int r = 1 + 1 + 99 + (static_cast<int>(sizeof(kRTaps) / sizeof(int)) - 1);
  int s = 2 + 98 + s_feedback_positions() + 1;
  return r + s + (mixing ? 3 : 1);
}

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F &&f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

}  // namespace mickey
