// decode_spa.cu -- the single-precision sum-product decoding kernel.
#include "decode_impl.cuh"

namespace tsx {
cudaError_t launch_spa(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                       cudaStream_t st) {
    return launch_scalar<DecSpa>(g, dp, b, sh, st);
}
}  // namespace tsx
