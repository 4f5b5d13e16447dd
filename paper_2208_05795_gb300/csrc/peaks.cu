// peaks.cu -- measure_peaks(): per-SM issue rates of the operations the
// decoders are built from, measured on the device the library runs on, so
// that a roofline can be stated against measured rather than nominal
// figures.  The paper has no counterpart.
//
// Each probe launches one CTA per resident slot (every SM full), runs a
// fixed number of independent operations per thread, and reads the SM's
// cycle counter (%clock64) at the start and end of every CTA.  The rate of
// an SM is (operations its CTAs executed) / (last end - first start) over
// its CTAs, in operations (or bytes) per SM clock; the reported figure is
// the median over SMs.  Every loop has a fixed trip count.
#include <algorithm>
#include <vector>

#include "kernels.cuh"

namespace {

constexpr int kThreads = 512;
constexpr int kIters = 4096;  // loop trips per thread
constexpr int kUnroll = 16;   // independent accumulators per thread

struct Span {
    long long t0, t1;
    int sm;
};

__device__ __forceinline__ int smid() {
    int s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

__device__ __forceinline__ void span_begin(long long &t0) {
    __syncthreads();
    t0 = clock64();
}
__device__ __forceinline__ void span_end(long long t0, Span *out) {
    __syncthreads();
    if (threadIdx.x == 0) out[blockIdx.x] = Span{t0, clock64(), smid()};
}

// 32-bit integer ALU: per step one min and one xor on each accumulator
// (neither pair can be merged into one instruction)
__global__ void __launch_bounds__(kThreads) int_probe(unsigned k1, unsigned k2, unsigned *sink, Span *sp) {
    unsigned a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = threadIdx.x * 2654435761u + u;
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            asm volatile("min.u32 %0, %0, %1;" : "+r"(a[u]) : "r"(k1));
            asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[u]) : "r"(k2));
        }
    }
    span_end(t0, sp);
    unsigned x = 0;
#pragma unroll
    for (int u = 0; u < kUnroll; u++) x ^= a[u];
    if (x == 0x12345678u) sink[0] = x;
}

// the packed 16-bit form of the same: min.u16x2 and xor
__global__ void __launch_bounds__(kThreads) u16x2_probe(unsigned k1, unsigned k2, unsigned *sink, Span *sp) {
    unsigned a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = threadIdx.x * 2654435761u + u;
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            asm volatile("min.u16x2 %0, %0, %1;" : "+r"(a[u]) : "r"(k1));
            asm volatile("xor.b32 %0, %0, %1;" : "+r"(a[u]) : "r"(k2));
        }
    }
    span_end(t0, sp);
    unsigned x = 0;
#pragma unroll
    for (int u = 0; u < kUnroll; u++) x ^= a[u];
    if (x == 0x12345678u) sink[0] = x;
}

// shared-memory loads: 16-byte vector loads, consecutive lanes on
// consecutive 16-byte words (no bank conflict), from a 32 KB buffer
__global__ void __launch_bounds__(kThreads) smem_probe(unsigned *sink, Span *sp) {
    __shared__ __align__(16) uint4 buf[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) buf[i] = make_uint4(i, i * 3, i * 5, i * 7);
    uint4 acc = make_uint4(0, 0, 0, 0);
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters / 4; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
            const unsigned idx = (threadIdx.x + (unsigned)u * 128u) & 2047u;
            uint4 v;
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "r"(base + idx * 16u));
            acc.x ^= v.x;
            acc.y ^= v.y;
            acc.z ^= v.z;
            acc.w ^= v.w;
        }
    }
    span_end(t0, sp);
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == 0x12345678u) sink[0] = acc.x;
}

// 32-bit integer multiply-add (mad.lo.u32 with register operands): the
// integer work the FMA pipe can take
__global__ void __launch_bounds__(kThreads) imad_probe(unsigned k1, unsigned k2, unsigned *sink, Span *sp) {
    unsigned a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = threadIdx.x * 2654435761u + u;
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[u]) : "r"(k1), "r"(k2));
    }
    span_end(t0, sp);
    unsigned x = 0;
#pragma unroll
    for (int u = 0; u < kUnroll; u++) x ^= a[u];
    if (x == 0x12345678u) sink[0] = x;
}

// the special-function unit: ex2.approx.f32
__global__ void __launch_bounds__(kThreads) sfu_probe(float *sink, Span *sp) {
    float a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = -1.0f - 1e-3f * (float)(threadIdx.x + u);
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters / 4; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) asm volatile("ex2.approx.f32 %0, %0;" : "+f"(a[u]));
    }
    span_end(t0, sp);
    float x = 0.0f;
#pragma unroll
    for (int u = 0; u < kUnroll; u++) x += a[u];
    if (x == 1234.5f) sink[0] = x;
}

// single-precision fused multiply-add
__global__ void __launch_bounds__(kThreads) fma_probe(float k1, float k2, float *sink, Span *sp) {
    float a[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; u++) a[u] = 1e-3f * (float)(threadIdx.x + u);
    long long t0;
    span_begin(t0);
    for (int it = 0; it < kIters; it++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[u]) : "f"(k1), "f"(k2));
    }
    span_end(t0, sp);
    float x = 0.0f;
#pragma unroll
    for (int u = 0; u < kUnroll; u++) x += a[u];
    if (x == 1234.5f) sink[0] = x;
}

// median over SMs of (per-CTA work x CTAs on the SM) / (SM's span in cycles)
double rate(const std::vector<Span> &sp, double work_per_cta, int num_sms) {
    std::vector<long long> lo(num_sms, -1), hi(num_sms, -1);
    std::vector<int> cnt(num_sms, 0);
    for (const Span &s : sp) {
        if (s.sm < 0 || s.sm >= num_sms) continue;
        lo[s.sm] = lo[s.sm] < 0 ? s.t0 : std::min(lo[s.sm], s.t0);
        hi[s.sm] = std::max(hi[s.sm], s.t1);
        cnt[s.sm]++;
    }
    std::vector<double> r;
    for (int i = 0; i < num_sms; i++)
        if (cnt[i] && hi[i] > lo[i]) r.push_back(work_per_cta * cnt[i] / (double)(hi[i] - lo[i]));
    if (r.empty()) return 0.0;
    std::sort(r.begin(), r.end());
    return r[r.size() / 2];
}

template <class K, class... A>
int run_probe(K k, int num_sms, cudaStream_t s, Span *d_sp, std::vector<Span> &h_sp, A... args) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, 0) != cudaSuccess || occ < 1)
        return TSX_ECUDA;
    const int blocks = occ * num_sms;
    h_sp.assign(blocks, Span{0, 0, -1});
    for (int rep = 0; rep < 2; rep++) {  // the first launch warms up; the second is measured
        k<<<blocks, kThreads, 0, s>>>(args..., d_sp);
        if (cudaGetLastError() != cudaSuccess) return TSX_ECUDA;
    }
    if (cudaMemcpyAsync(h_sp.data(), d_sp, sizeof(Span) * blocks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return TSX_ECUDA;
    return TSX_OK;
}

}  // namespace

extern "C" int measure_peaks(tsx_peaks *out, void *stream) {
    if (!out) return TSX_EINVAL;
    *out = tsx_peaks{};
    int dev = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || num_sms < 1)
        return TSX_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int max_blocks = 64 * num_sms;
    Span *d_sp = nullptr;
    unsigned *sink = nullptr;
    if (cudaMalloc(&d_sp, sizeof(Span) * max_blocks) != cudaSuccess) return TSX_ENOMEM;
    if (cudaMalloc(&sink, 16) != cudaSuccess) {
        cudaFree(d_sp);
        return TSX_ENOMEM;
    }
    std::vector<Span> h;
    const double thr_ops = (double)kThreads * kIters * kUnroll;
    int st = TSX_OK;
    out->num_sms = num_sms;
    if ((st = run_probe(int_probe, num_sms, s, d_sp, h, 0x7fffffffu, 0x5bd1e995u, sink)) == TSX_OK)
        out->int32_ops_per_clk_sm = rate(h, 2.0 * thr_ops, num_sms);
    if (st == TSX_OK && (st = run_probe(u16x2_probe, num_sms, s, d_sp, h, 0x7fff7fffu, 0x5bd1e995u, sink)) == TSX_OK)
        out->u16x2_ops_per_clk_sm = rate(h, 2.0 * thr_ops, num_sms);
    if (st == TSX_OK && (st = run_probe(smem_probe, num_sms, s, d_sp, h, sink)) == TSX_OK)
        out->smem_bytes_per_clk_sm = rate(h, 16.0 * thr_ops / 4, num_sms);
    if (st == TSX_OK && (st = run_probe(sfu_probe, num_sms, s, d_sp, h, (float *)sink)) == TSX_OK)
        out->sfu_ops_per_clk_sm = rate(h, thr_ops / 4, num_sms);
    if (st == TSX_OK && (st = run_probe(fma_probe, num_sms, s, d_sp, h, 0.999f, 1e-4f, (float *)sink)) == TSX_OK)
        out->fp32_fma_per_clk_sm = rate(h, thr_ops, num_sms);
    if (st == TSX_OK && (st = run_probe(imad_probe, num_sms, s, d_sp, h, 0x9E3779B9u, 0x7F4A7C15u, sink)) == TSX_OK)
        out->imad_ops_per_clk_sm = rate(h, thr_ops, num_sms);
    cudaStreamSynchronize(s);
    cudaFree(d_sp);
    cudaFree(sink);
    return st;
}
