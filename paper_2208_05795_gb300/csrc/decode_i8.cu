// decode_i8.cu -- instantiation of the decoding kernel for DecNms8.
#include "decode_impl.cuh"

namespace tsx {
cudaError_t launch_enum_i8(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                            const LaunchShape &sh, cudaStream_t st) {
    return launch_dec<DecNms8>(g, dp, b, sh, st);
}
}  // namespace tsx
