// Persistent keystream kernels with ST = 4: two blocks per SM (two warps per SM sub-partition), rows staged 4 tiles.
#include "keystream_persistent.cuh"

namespace mickey {

cudaError_t launch_persistent4(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                               const PersistArgs &p, cudaStream_t st) {
  return launch_persistent_st<4>(a, layout, unroll, e, p, st);
}

}  // namespace mickey
