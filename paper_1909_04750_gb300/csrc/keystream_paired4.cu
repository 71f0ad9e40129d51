// Paired clock/emission keystream kernels with rows staged ST = 4 tiles
// deep (one block per SM; tuner candidates beside the ST = 8 kernel).
#include "keystream_persistent.cuh"

namespace mickey {

cudaError_t launch_paired4(const KeystreamArgs &a, int layout, int unroll, const EmitCtx &e,
                           const PersistArgs &p, cudaStream_t st) {
  return launch_ws_st<4>(a, layout, unroll, e, p, st);
}

}  // namespace mickey
