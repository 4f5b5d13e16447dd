// decode_i16.cu -- instantiation of the decoding kernel for DecNms16.
#include "decode_impl.cuh"

namespace tsx {
cudaError_t launch_enum_i16(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                            const LaunchShape &sh, cudaStream_t st) {
    return launch_dec<DecNms16>(g, dp, b, sh, st);
}
}  // namespace tsx
