// noalloc.cu -- decode_thresholds_noalloc(): the impulse-decoding kernel run
// on caller-given candidate sets with all of its working memory in one
// fixed device array, for callers that cannot allocate device memory (a
// host thread that must not take the driver's allocation locks, code running
// under another framework's memory manager that forbids outside cudaMalloc,
// or a process that has reserved the whole device).  The call does wait for
// its stream once, for the device-side check of the candidate sets.  The
// paper has no counterpart; the decoding is the same kernel enumerate_ts()
// uses.
#include <mutex>

#include "kernels.cuh"

namespace {

// Working memory of decode_thresholds_noalloc: the decoder's work-queue and
// statistics counters, a checked copy of the candidate sets, the float
// thresholds / table slots / flags the decoder writes for every candidate,
// and the x* patterns it writes for failing ones.  Every GPU that loads the
// library holds these TSX_NOALLOC_SCRATCH_BYTES until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[TSX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];  // device address of g_noalloc_scratch, per device

// The array's device address for the current device (looked up once per
// device; the host-side name of the array is not a device address).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSX_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return TSX_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TSX_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TSX_OK;
}

// Copies the candidate sets into the scratch and counts malformed ones: an
// entry outside [0, n), a -1 before a valid entry, or an empty set.
__global__ void check_cands_kernel(const int4 *in, long long n_cand, int n, int4 *out, unsigned *bad,
                                   tsx::Counters *ctr) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_cand_total = (unsigned long long)n_cand;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_cand;
         i += (long long)gridDim.x * blockDim.x) {
        const int4 c = in[i];
        const int v[4] = {c.x, c.y, c.z, c.w};
        bool ok = v[0] >= 0;
        bool ended = false;
        for (int k = 0; k < 4; k++) {
            if (v[k] < 0) {
                ended = true;
                ok = ok && v[k] == -1;
            } else {
                ok = ok && !ended && v[k] < n;
            }
        }
        out[i] = ok ? c : make_int4(-1, -1, -1, -1);
        if (!ok) atomicAdd(bad, 1u);
    }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

using namespace tsx;

extern "C" int decode_thresholds_noalloc(const tsx_code *code, const tsx_enum_params *params,
                                         const int32_t *cand_vars, int64_t n_cand, int32_t *thr, float *thr_f,
                                         int32_t *decodes, int32_t *iters, void *stream) {
    if (!code || !params || n_cand < 0) return TSX_EINVAL;
    if (n_cand == 0) return TSX_OK;
    if (!cand_vars || !thr || !decodes || !iters) return TSX_EINVAL;
    if (((uintptr_t)cand_vars & 15) != 0) return TSX_EINVAL;
    DecodeParams dp;
    int st = enum_params_to_decode(params, &dp);
    if (st != TSX_OK) return st;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return TSX_ECUDA;
    if (dev != code_device(code)) return TSX_EINVAL;
    const DevCode &g = *code_dev(code);
    const int nw = (g.n + 31) / 32;
    // 28 + 4 nw bytes per candidate: refuse a count beyond the array before
    // any size arithmetic can wrap
    if ((uint64_t)n_cand > (uint64_t)TSX_NOALLOC_SCRATCH_BYTES / (28u + 4u * (uint64_t)nw)) return TSX_ENOMEM;
    // carve: counters | bad flag | checked sets | thr_f | slot | flags | x*
    const size_t off_bad = al256(sizeof(Counters));
    const size_t off_cands = al256(off_bad + sizeof(unsigned));
    const size_t off_thrf = al256(off_cands + (size_t)n_cand * 16);
    const size_t off_slot = al256(off_thrf + (size_t)n_cand * 4);
    const size_t off_flags = al256(off_slot + (size_t)n_cand * 4);
    const size_t off_x = al256(off_flags + (size_t)n_cand * 4);
    const size_t need = off_x + (size_t)n_cand * nw * 4;
    if (need > (size_t)TSX_NOALLOC_SCRATCH_BYTES) return TSX_ENOMEM;
    void *base = nullptr;
    st = scratch_address(&base);
    if (st != TSX_OK) return st;
    unsigned char *sc = (unsigned char *)base;
    cudaStream_t s = (cudaStream_t)stream;

    // the previous call's contents are still there: zero the counters (the
    // queue head and statistics) and the malformed-set count
    if (cudaMemsetAsync(sc, 0, off_cands, s) != cudaSuccess) return TSX_ECUDA;
    int blocks = (int)((n_cand + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    check_cands_kernel<<<blocks, 256, 0, s>>>((const int4 *)cand_vars, n_cand, g.n, (int4 *)(sc + off_cands),
                                             (unsigned *)(sc + off_bad), (Counters *)sc);
    if (cudaGetLastError() != cudaSuccess) return TSX_ECUDA;
    unsigned bad = 0;
    if (cudaMemcpyAsync(&bad, sc + off_bad, sizeof(bad), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TSX_ECUDA;
    if (bad) return TSX_EINVAL;

    EnumBuffers b{};
    b.cands = (const int4 *)(sc + off_cands);
    b.cand_begin = 0;
    b.cand_end = n_cand;
    b.record = 1;
    b.c_thr = thr;
    b.c_thr_f = thr_f ? thr_f : (float *)(sc + off_thrf);
    b.c_slot = (int *)(sc + off_slot);
    b.c_flags = (int *)(sc + off_flags);
    b.c_decodes = decodes;
    b.c_iters = iters;
    b.xstar = (uint32_t *)(sc + off_x);
    b.nw = nw;
    b.ctr = (Counters *)sc;
    b.queue = &b.ctr->next_cand;
    b.rec_base = 0;
    if (launch_decode(g, dp, b, params->warps_per_cta, 0, params->ctas_per_sm, code_num_sms(code),
                      params->kernel == 1 ? 1 : 0, s) != cudaSuccess)
        return TSX_ECUDA;
    return TSX_OK;
}
