// decode_i8.cu -- the min-sum decoding kernels with int8 message storage.
#include "decode_pair.cuh"

namespace tsx {
cudaError_t launch_nms8(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                         bool pair, cudaStream_t st) {
    if (pair) return launch_pair<true>(g, dp, b, sh, st);
    return launch_scalar<DecNms8>(g, dp, b, sh, st);
}
}  // namespace tsx
