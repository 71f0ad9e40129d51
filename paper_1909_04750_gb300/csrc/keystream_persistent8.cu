// Persistent keystream kernels with ST = 8: one block per SM (four clock
// warps and four emission warps), rows staged in whole 32-byte sectors.
#include "keystream_persistent.cuh"

namespace mickey {

cudaError_t launch_persistent8(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                               const PersistArgs &p, cudaStream_t st) {
  return launch_ws_st<8>(a, layout, unroll, e, p, st);
}

}  // namespace mickey
