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
// and caches it with the id of the device's context; after a cudaDeviceReset
// the next call finds a new context and looks the address up again.  That
// first call (and the first call after a reset) must therefore come before
// any stream capture on the device.  All calls share the one array and it keeps the
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
unsigned long long g_ctx[kMaxDevices] = {};

// Id of the calling thread's current CUDA context (0 if it cannot be told).
// Context ids are never reused within a process, so a context rebuilt after
// cudaDeviceReset gets a new one.  The driver calls are reached through the
// runtime's entry-point lookup, so the library needs no libcuda link.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(f);
      get_id = reinterpret_cast<GetId>(g);
    }
  });
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// The array's device address on the current device, looked up with that
// device current the first time and again whenever the device's context has
// changed since (cudaDeviceReset rebuilds the context and may move the
// array).  If the context cannot be identified it is looked up every call.
int scratch_address(uint32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(MICKEY_E_CUDA, "no usable current CUDA device");
  std::lock_guard<std::mutex> lock(g_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(MICKEY_E_CUDA, "cudaGetSymbolAddress of the fixed scratch array failed");
    g_addr[dev] = static_cast<uint32_t *>(p);
    g_ctx[dev] = current_context_id();   // the lookup has made the context current
  }
  *out = g_addr[dev];
  return MICKEY_OK;
}

}  // namespace

extern "C" MICKEY_API int mickey_init_state_noalloc(const uint8_t *keys, const uint8_t *ivs,
                                                    const uint32_t *iv_lens, size_t n,
                                                    uint32_t *state, void *cuda_stream) {
  if (!keys || !ivs || !state || n == 0)
    return set_error(MICKEY_E_ARG, "keys, ivs and state must not be NULL and n must be > 0");
  if (n > kMaxStreams)
    return set_error(MICKEY_E_ARG, "n is above MICKEY_NOALLOC_MAX_STREAMS (the fixed array)");
  if (iv_lens)
    for (size_t i = 0; i < n; ++i)
      if (iv_lens[i] > MICKEY_MAX_IV_BITS)
        return set_error(MICKEY_E_IVLEN, "an IV length exceeds 80 bits");
  uint32_t *base = nullptr;
  if (const int rc = scratch_address(&base)) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const uint32_t G = uint32_t((n + 31) / 32), Gpad = (G + 31u) & ~31u;
  uint8_t *in = reinterpret_cast<uint8_t *>(base + kInputWords);
  // The load kernel raises this flag only for an IV length above 80, which
  // the host has ruled out above, so the word needs no clearing.
  int *err = reinterpret_cast<int *>(base + kErrWord);
  uint32_t *rows = base + kRowsWord;
  // every scratch row the kernels read is written by this call's load kernel
  if (cudaMemcpyAsync(in, keys, n * 10, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(in + n * 10, ivs, n * 10, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "copy of keys and IVs into the fixed array failed");
  const uint32_t *lens = nullptr;
  if (iv_lens) {
    if (cudaMemcpyAsync(in + n * 20, iv_lens, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return set_error(MICKEY_E_CUDA, "copy of IV lengths into the fixed array failed");
    lens = reinterpret_cast<const uint32_t *>(in + n * 20);
  }
  LoadArgs la{in, in + n * 10, lens, n, nullptr, G, Gpad, rows, err};
  if (launch_init(la, state, st) != cudaSuccess)
    return set_error(MICKEY_E_CUDA, "init_kernel launch");
  return set_error(MICKEY_OK, "");
}
