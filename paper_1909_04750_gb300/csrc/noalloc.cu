// mickey_init_state_noalloc: key/IV loading and preclocking that allocates
// no device memory.
//
// Who needs it: code that is not allowed to call cudaMalloc/cudaFree --
// e.g. a plug-in running inside a host application whose own allocator owns
// all device memory, or a latency-critical loop that must not hit the
// implicit device synchronisation of cudaFree or the cost of a fresh
// allocation.  Such callers pass their inputs and an output buffer they
// already own; the temporary memory the key/IV bitslicing needs lives in a
// fixed-size array of this library instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 3.6 MB) until the process exits.  Host code may not
// use the variable's name as an address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it.  That first call must therefore come before any stream
// capture on the device.  All calls share the one array and it keeps the
// previous call's contents, so two calls whose work overlaps on the GPU
// (for example on two streams) race with each other: serialise them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/mickey.h"
#include "internal.h"

namespace {

using namespace mickey;

constexpr size_t kMaxStreams = MICKEY_NOALLOC_MAX_STREAMS;
constexpr size_t kMaxGroupsPad = ((kMaxStreams + 31) / 32 + 31) / 32 * 32;
// word offsets inside the array
constexpr size_t kErrWord = 0;
constexpr size_t kInputWords = 64;                       // keys, ivs, lens
constexpr size_t kInputBytes = kMaxStreams * 24;
constexpr size_t kRowsWord = kInputWords + kInputBytes / 4;
constexpr size_t kTotalWords = kRowsWord + size_t(kScratchRows + 1) * kMaxGroupsPad;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kTotalWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t *g_addr[kMaxDevices] = {};

// The array's device address on the current device (looked up once).
int scratch_address(uint32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MICKEY_E_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MICKEY_E_CUDA;
    g_addr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_addr[dev];
  return MICKEY_OK;
}

}  // namespace

extern "C" MICKEY_API int mickey_init_state_noalloc(const uint8_t *keys, const uint8_t *ivs,
                                                    const uint32_t *iv_lens, size_t n,
                                                    uint32_t *state, void *cuda_stream) {
  if (!keys || !ivs || !state || n == 0) return MICKEY_E_ARG;
  if (n > kMaxStreams) return MICKEY_E_ARG;  // beyond the fixed array
  if (iv_lens)
    for (size_t i = 0; i < n; ++i)
      if (iv_lens[i] > MICKEY_MAX_IV_BITS) return MICKEY_E_IVLEN;
  uint32_t *base = nullptr;
  if (scratch_address(&base) != MICKEY_OK) return MICKEY_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const uint32_t G = uint32_t((n + 31) / 32), Gpad = (G + 31u) & ~31u;
  uint8_t *in = reinterpret_cast<uint8_t *>(base + kInputWords);
  int *err = reinterpret_cast<int *>(base + kErrWord);
  uint32_t *rows = base + kRowsWord;
  // the error word must start at zero; every scratch row the kernels read
  // is written by the load kernel of this call first
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess ||
      cudaMemcpyAsync(in, keys, n * 10, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(in + n * 10, ivs, n * 10, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return MICKEY_E_CUDA;
  const uint32_t *lens = nullptr;
  if (iv_lens) {
    if (cudaMemcpyAsync(in + n * 20, iv_lens, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return MICKEY_E_CUDA;
    lens = reinterpret_cast<const uint32_t *>(in + n * 20);
  }
  LoadArgs la{in, in + n * 10, lens, n, nullptr, G, Gpad, rows, err};
  if (launch_load(la, st) != cudaSuccess) return MICKEY_E_CUDA;
  PreclockArgs pa{rows, state, G, Gpad};
  if (launch_preclock(pa, st) != cudaSuccess) return MICKEY_E_CUDA;
  return MICKEY_OK;
}
