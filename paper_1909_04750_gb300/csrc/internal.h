// Internal interfaces between the C ABI (capi.cu) and the kernel
// translation units.  Plain pointers and sizes only.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace mickey {

// Device-side error bits, OR-ed into a per-handle flag word.
constexpr int kErrIvLen = 1;
constexpr int kErrTimeout = 2;

// Rows of the bitsliced input scratch, each Gpad words long:
//   [0, 80)    key words K[j], bit l = key bit j of lane l
//   [80, 160)  IV-phase input words, right-aligned per lane
//   [160, 240) IV-phase activity masks (only read for mixed-length groups)
// followed by one info word per group: max IV length | (mixed << 8).
constexpr int kKeyRow = 0;
constexpr int kIvRow = 80;
constexpr int kActRow = 160;
constexpr int kScratchRows = 240;

// Bitsliced state: 200 rows of Gpad words, r0..r99 then s0..s99.
constexpr int kStateRows = 200;

constexpr int kInitThreads = 128;

struct LoadArgs {
  const uint8_t *keys;      // n x 10, device
  const uint8_t *ivs;       // n x 10, device
  const uint32_t *iv_lens;  // n, device, or nullptr (= 80)
  uint64_t n;
  const uint32_t *perm;     // lane slot -> instance, or nullptr (identity)
  uint32_t G, Gpad;
  uint32_t *scratch;        // kScratchRows * Gpad + Gpad words
  int *err;
};

// Key/IV loading and preclocking of every group (init_kernels.cu): the
// scratch rows of `a`, then the 200-word state into `state` (kStateRows *
// Gpad words).
cudaError_t launch_init(const LoadArgs &a, uint32_t *state, cudaStream_t st);

struct KeystreamArgs {
  uint32_t *state;          // kStateRows * Gpad words, read and written back
  uint32_t G, Gpad;
  uint64_t n;               // instances
  uint64_t n_bits;          // keystream bits per instance in this call
  void *out;                // device output, layout-dependent
};

// Record the thread-local error reported by mickey_last_error (code 0
// clears it); returns `code`.
int set_error(int code, const char *msg);

}  // namespace mickey
struct mickey_streams;
namespace mickey {
// Device state words of a handle (kStateRows x Gpad, word-major).
const uint32_t *handle_state(const mickey_streams *s, uint32_t *G, uint32_t *Gpad);

// Unroll factors compiled for the keystream kernel.
constexpr int kUnrolls[] = {2, 4};
// Largest n_bits of one keystream launch: a row of the row-major layouts
// must stay below 4 GiB.
constexpr uint64_t kMaxBitsPerCall = 1ull << 34;
constexpr int kKsThreads = 128;

// Persistent mode (see keystream_persistent_kernel): W warp-groups, L tiles
// per warp, one flag word per warp-group (compared with `epoch`).
struct PersistArgs {
  uint32_t blocks;      // grid: 1 or 2 blocks per SM (cooperative), or one block per
                        // 4 warp-groups (paired launch with L = NT, not cooperative)
  uint32_t cooperative; // 1: all blocks resident (needed when segments hand off)
  uint32_t stage_tiles; // row staging depth in tiles: 2, 4 or 8 (paired kernel), 4 (two-block)
  uint32_t paired;      // 1: clock warps paired with emission warps; 0: two-block kernel
  uint32_t W;           // warp-groups = ceil(G / 32)
  uint64_t L;           // tiles of the work line per warp
  uint32_t *flags;      // W words
  uint32_t epoch;       // value a finished head piece writes
  uint32_t wait_epoch;  // value a tail piece waits for (== epoch; differs only under the
                        // MICKEY_TEST_UNPUBLISHED test hook, to make the wait run out)
  uint32_t spin_limit;  // bounded wait of a tail piece (iterations of ~256 ns)
  int *err;
};

// Ragged generation on a handle (ragged.cu): stream i continues by
// n_bits[i] bits; its output starts at byte offsets[i] of out (row layouts)
// or, for the bitsliced layout, group g's words start at offsets[g].
struct RaggedArgs {
  uint32_t *state;          // kStateRows * Gpad words, read and written back
  uint32_t G, Gpad;
  uint64_t n;
  const uint64_t *n_bits;   // n values, device
  const uint64_t *offsets;  // n (row layouts) or G (bitsliced) byte offsets, device
  uint8_t *out;
};
cudaError_t launch_ragged(const RaggedArgs &a, int layout, cudaStream_t st);

// p == nullptr: grid mode (one thread per group); else persistent mode.
// stage: row layouts stage this many tiles per row (grid: 2 or 4; persistent:
// p->stage_tiles) and write whole chunks of 4 x stage bytes per row, used when
// n_bits is a multiple of 32 x stage and `out` is 16-byte aligned; 0: direct
// 4-byte row stores.
cudaError_t launch_keystream(const KeystreamArgs &a, int layout, int unroll, int stage,
                             const PersistArgs *p, cudaStream_t st);

}  // namespace mickey
