// decode_spa.cu -- instantiation of the decoding kernel for DecSpa.
#include "decode_impl.cuh"

namespace tsx {
cudaError_t launch_enum_spa(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                            const LaunchShape &sh, cudaStream_t st) {
    return launch_dec<DecSpa>(g, dp, b, sh, st);
}
}  // namespace tsx
