// decode_i8.cu -- the min-sum decoding kernels with int8 message storage.
#include "decode_pair.cuh"

namespace tsx {
cudaError_t launch_nms8(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                         bool pair, cudaStream_t st) {
    if (pair) return launch_pair<true>(g, dp, b, sh, st);
    return launch_scalar<DecNms8>(g, dp, b, sh, st);
}
cudaError_t launch_batch8(const BatchArgs &items, int n, bool qc, int dc_max, bool reg6, const LaunchShape &sh,
                           cudaStream_t st) {
    return launch_batch_t<true>(items, n, qc, dc_max, reg6, sh, st);
}
}  // namespace tsx
