// decode_i16.cu -- the min-sum decoding kernels with int16 message storage.
#include "decode_pair.cuh"

namespace tsx {
cudaError_t launch_nms16(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                         bool pair, cudaStream_t st) {
    if (pair) return launch_pair<false>(g, dp, b, sh, st);
    return launch_scalar<DecNms16>(g, dp, b, sh, st);
}
// the variable-node-pass form of the two-codeword kernel (QC, check degree > 8)
cudaError_t launch_nms16_vn(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                            cudaStream_t st) {
    return launch_persistent(pair_vn_kernel<false>, sh, st, g, dp, b, sh.lay, sh.G);
}
cudaError_t launch_batch16(const BatchArgs &items, int n, bool qc, int dc_max, bool reg6, const LaunchShape &sh,
                           cudaStream_t st) {
    return launch_batch_t<false>(items, n, qc, dc_max, reg6, sh, st);
}
}  // namespace tsx
