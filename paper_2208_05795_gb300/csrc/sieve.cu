// sieve.cu -- the sieve kernel: Tree()/TS() extraction, (a,b), canonical
// key, orbit and hash insert of every failing candidate.
#include "decode_impl.cuh"

namespace tsx {
cudaError_t launch_sieve_kernel(const DevCode &g, const EnumBuffers &b, const LaunchShape &sh, int is_float,
                                cudaStream_t st) {
    if (g.kind == TSX_CODE_QC) return launch_persistent(sieve_kernel<true>, sh, st, g, b, sh.lay, is_float);
    return launch_persistent(sieve_kernel<false>, sh, st, g, b, sh.lay, is_float);
}
}  // namespace tsx
