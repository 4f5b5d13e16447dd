// isfer.cu -- importance-sampling FER toward a trapping set (the weighting
// step the paper takes from Cole, Sec. II-III): mean-shift importance
// sampling of BPSK over AWGN, with the noise on the set's bits shifted by
// -mu, every sample decoded by the fixed-point min-sum decoder, and
//   FER = mean over samples of fail * w,
//   log w = sum_{v in T, ascending} (n_v mu / sigma^2 - mu^2 / (2 sigma^2)).
// Noise: Philox4x32-10 (Salmon et al., SC'11) keyed by the job, counter
// (v / 4, sample low, sample high, 0); uniforms u = (2 (x >> 9) + 1) 2^-24;
// Box-Muller pairs in single precision with IEEE-rounded operations only
// (log by frexp and the atanh series; sin/cos of 2 pi u by quadrant
// reduction and Taylor series on [0, pi/4]); channel LLR quantized as
// round-half-away(8 * 2 y / sigma^2) saturated to +-sat.  Log-weights in
// double precision; the sums are reduced in a fixed order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "decode_pair.cuh"
#include "noise.cuh"

namespace tsx {
namespace {

struct IsArgs {
    unsigned long long job, s0;
    long long nsamp;
    float sigf, muf, cq;
    double A, Bc;
    const int *T;
    int a;
    double *wfail;            // [nsamp] fail * w
    unsigned char *fail_out;  // [nsamp] or null
    double *logw_out;         // [nsamp] or null
    Counters *ctr;
    unsigned long long *queue;  // work-queue word of this launch (samples s0 + i, i < nsamp)
};

// ---------------------------------------------------------------------------
// the sampling kernel: two samples per lane, as the enumeration decoder
// ---------------------------------------------------------------------------
// QC codes of check degree > 8 run the check pass over all row blocks at once
// (FLAT), so that one sample pair can take more warps than Z / 32.
template <bool QC, int DC, bool EXACT>
__global__ void __launch_bounds__(QC && DC > 8 ? 32 * kIsWarps : 512) is_kernel(DevCode g, DecodeParams dp, IsArgs ia,
                                                                               SlotLayout lay, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem, true);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = warp / G;
    unsigned char *slot = smem + lay.tables_bytes + grp * lay.slot_bytes;
    Misc *misc = (Misc *)(slot + lay.misc_off);
    Grp gp;
    gp.G = G;
    gp.T = 32 * G;
    gp.gw = warp - grp * G;
    gp.gt = gp.gw * 32 + lane;
    gp.lane = lane;
    gp.bar = 1 + grp;
    gp.red = misc->red;
    unsigned char *Rb = slot + lay.r_off;
    unsigned *Pbuf = (unsigned *)(slot + lay.p_off);  // [2][n]
    unsigned *L2 = Pbuf + 2 * g.n;                    // accumulator start values, both halves
    uint32_t *Tm = (uint32_t *)(slot + lay.xa_off);   // bitmask of T
    const int nw = (g.n + 31) >> 5;

    PairConst pc;
    pc.B = 1024;
    pc.sat = dp.sat;
    pc.an = dp.alpha_num;
    pc.as = dp.alpha_shift;
    pc.B2 = (unsigned)pc.B * 0x00010001u;
    pc.BETA2 = kBeta * 0x00010001u;
    pc.BS2 = (kBeta + (unsigned)pc.sat) * 0x00010001u;
    pc.amask2 = (0xFFFFu >> pc.as) * 0x00010001u;
    pc.BAN2 = pc.BETA2 * (unsigned)pc.an;
    // QC codes: the all-row-block pass for check degree > 8 (wider groups) and for
    // degree 7-8 (the row block's shifts read from the tables, not held in registers)
    PairDecoder<QC, DC, EXACT, false, false, QC && (DC > 8 || !EXACT)> dec{g, sg, gp, pc, Rb};

    for (int w = gp.gt; w < nw; w += gp.T) Tm[w] = 0u;
    gp.sync();
    for (int t = gp.gt; t < ia.a; t += gp.T) atomicOr(&Tm[ia.T[t] >> 5], 1u << (ia.T[t] & 31));
    gp.sync();

    long long my_dec = 0, my_it = 0;
    long long sidx[2];
    int k[2], first[2];
    int pcur = 0;

    auto fetch = [&](int hh) {
        if (gp.gt == 0) misc->bcast[0] = (long long)atomicAdd(ia.queue, 1ull);
        gp.sync();
        const long long i = misc->bcast[0];
        gp.sync();
        sidx[hh] = i < ia.nsamp ? i : -1;
        k[hh] = 0;
        first[hh] = 1;
    };
    // channel values of sample sidx[hh] into half hh of L2 (accumulator
    // start) and of the current posteriors (P = L); an idle half gets L = 0
    auto generate = [&](int hh, unsigned *Pc) {
        const unsigned long long s = ia.s0 + (unsigned long long)(sidx[hh] < 0 ? 0 : sidx[hh]);
        for (int q = gp.gt; 4 * q < g.n; q += gp.T) {
            float gq[4];
            if (sidx[hh] >= 0) normals4(ia.job, s, (uint32_t)q, gq);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int v = 4 * q + j;
                if (v >= g.n) break;
                int L = 0;
                if (sidx[hh] >= 0) {
                    const float n = hmul(ia.sigf, gq[j]);
                    float y = hadd(1.0f, n);
                    if ((Tm[v >> 5] >> (v & 31)) & 1u) y = hsub(y, ia.muf);
                    const float lq = roundf(hmul(y, ia.cq));
                    L = lq > (float)dp.sat ? dp.sat : (lq < -(float)dp.sat ? -dp.sat : (int)lq);
                }
                dec.set_half(L2, v, hh, (unsigned)(L + (int)kBeta - dec.vdeg(v) * pc.B));
                dec.set_half(Pc, v, hh, (unsigned)(L + (int)kBeta));
            }
        }
    };

    {
        unsigned *Pc = Pbuf;
        for (int hh = 0; hh < 2; hh++) {
            fetch(hh);
            generate(hh, Pc);
        }
        gp.sync();
    }
    while (sidx[0] >= 0 || sidx[1] >= 0) {
        unsigned *Pc = Pbuf + pcur * g.n, *Pn = Pbuf + (pcur ^ 1) * g.n;
        if ((g.n & 3) == 0) {  // 16-byte copies (Pbuf is 16-byte aligned, so are Pn and L2)
            const uint4 *src = (const uint4 *)L2;
            uint4 *dst = (uint4 *)Pn;
            for (int q = gp.gt; q < (g.n >> 2); q += gp.T) dst[q] = src[q];
        } else {
            for (int v = gp.gt; v < g.n; v += gp.T) Pn[v] = L2[v];
        }
        gp.sync();
        const unsigned km = (first[0] ? 0xFFFF0000u : 0xFFFFFFFFu) & (first[1] ? 0x0000FFFFu : 0xFFFFFFFFu);
        const unsigned kb = pc.B2 & ~km;
        const bool wr = (sidx[0] >= 0 && k[0] < dp.K) || (sidx[1] >= 0 && k[1] < dp.K);
        // (the common form -- no half starting, messages written -- compiled with writeR constant)
        const int us = km != 0xFFFFFFFFu ? dec.template check_pass<true>(km, kb, wr, Pc, Pn)
                       : wr              ? dec.template check_pass<false>(km, kb, true, Pc, Pn)
                                         : dec.template check_pass<false>(km, kb, false, Pc, Pn);
        int restart[2] = {0, 0};
        for (int hh = 0; hh < 2; hh++) {
            if (sidx[hh] < 0) continue;
            const int u = hh == 0 ? (us & 0xFFFF) : (us >> 16);
            if (u != 0 && k[hh] != dp.K) continue;
            const bool fail = u != 0 || dec.any_neg(Pc, hh) != 0;
            if (gp.gt == 0) {
                const unsigned long long s = ia.s0 + (unsigned long long)sidx[hh];
                double lw = 0.0;
                for (int t = 0; t < ia.a; t++) {
                    const int v = ia.T[t];
                    float gq[4];
                    normals4(ia.job, s, (uint32_t)(v >> 2), gq);
                    const double n = (double)hmul(ia.sigf, gq[v & 3]);
                    lw = __dadd_rn(lw, __dsub_rn(__dmul_rn(n, ia.A), ia.Bc));
                }
                ia.wfail[sidx[hh]] = fail ? exp(lw) : 0.0;
                if (fail) atomicAdd(&ia.ctr->n_fail, 1ull);
                if (ia.fail_out) ia.fail_out[sidx[hh]] = fail ? 1 : 0;
                if (ia.logw_out) ia.logw_out[sidx[hh]] = lw;
            }
            my_dec++;
            my_it += k[hh];
            restart[hh] = 1;
        }
        gp.sync();
        for (int hh = 0; hh < 2; hh++) {
            if (restart[hh]) {
                fetch(hh);
                if (sidx[hh] >= 0) generate(hh, Pn);
            } else if (sidx[hh] >= 0) {
                k[hh]++;
                first[hh] = 0;
            }
        }
        gp.sync();
        pcur ^= 1;
    }
    if (gp.gt == 0) {
        atomicAdd(&ia.ctr->decodes, (unsigned long long)my_dec);
        atomicAdd(&ia.ctr->iterations, (unsigned long long)my_it);
        atomicAdd(&ia.ctr->edge_updates, (unsigned long long)my_it * (unsigned long long)g.E);
    }
}

// fixed-order reduction: per block, 4096 consecutive samples
constexpr int kRedBlock = 1024, kRedChunk = 4096;
__global__ void __launch_bounds__(kRedBlock) reduce_kernel(const double *w, long long n, double *part) {
    __shared__ double s1[kRedBlock], s2[kRedBlock];
    const long long base = (long long)blockIdx.x * kRedChunk;
    double a = 0.0, b = 0.0;
    for (int j = 0; j < kRedChunk / kRedBlock; j++) {
        const long long i = base + (long long)threadIdx.x * (kRedChunk / kRedBlock) + j;
        const double x = i < n ? w[i] : 0.0;
        a = __dadd_rn(a, x);
        b = __dadd_rn(b, __dmul_rn(x, x));
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int h = kRedBlock / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s1[threadIdx.x] = __dadd_rn(s1[threadIdx.x], s1[threadIdx.x + h]);
            s2[threadIdx.x] = __dadd_rn(s2[threadIdx.x], s2[threadIdx.x + h]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}
__global__ void finish_kernel(const double *part, int nb, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; i++) {
        a = __dadd_rn(a, part[2 * i]);
        b = __dadd_rn(b, part[2 * i + 1]);
    }
    out[0] = a;
    out[1] = b;
}

}  // namespace
}  // namespace tsx

using namespace tsx;

extern "C" void is_params_default(tsx_is_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->ebn0_db = 4.0;
    p->rate = 0.0;
    p->mu = 1.0;
    p->n_samples = 100000;
    p->job_key = 0;
    p->sample_begin = 0;
    p->K = 20;
    p->sat = 511;
    p->alpha_num = 3;
    p->alpha_shift = 2;
}

// ---------------------------------------------------------------------------
// jobs: validation and sizing, enqueue, collection
// ---------------------------------------------------------------------------
namespace tsx {

struct IsJob {
    DevCode g;
    DecodeParams dp{};
    LaunchShape sh{};
    IsArgs ia{};
    long long N = 0, chunk = 0, n_chunks = 0;
    int nb = 0, grid_sms = 0;
    std::vector<int> Ts;
    size_t off_p = 0, off_o = 0, off_q = 0, total = 0;
    unsigned char *B = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
};

static int is_plan(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p, long long chunk,
                   IsJob &J) {
    if (!code || !p || a < 0 || (a > 0 && !ts_vars)) return TSX_EINVAL;
    if (p->n_samples < 0 || p->sample_begin < 0 || p->K < 0 || p->K > 100000) return TSX_EINVAL;
    if (p->sat < 1 || p->sat > 8191 || p->alpha_shift < 0 || p->alpha_shift > 15 || p->alpha_num < 1 ||
        p->alpha_num > (1 << p->alpha_shift))
        return TSX_EINVAL;
    const DevCode &g = *code_dev(code);
    for (int t = 0; t < a; t++)
        if (ts_vars[t] < 0 || ts_vars[t] >= g.n) return TSX_EINVAL;
    const double rate = p->rate > 0.0 ? p->rate : 1.0 - (double)g.m / (double)g.n;
    if (!(rate > 0.0) || !(p->ebn0_db > -100.0 && p->ebn0_db < 100.0)) return TSX_EINVAL;
    J.g = g;
    J.dp.decoder = TSX_DEC_NMS_I16;
    J.dp.K = p->K;
    J.dp.sat = p->sat;
    J.dp.alpha_num = p->alpha_num;
    J.dp.alpha_shift = p->alpha_shift;
    J.dp.base_llr = 1;
    if (!plan_is_shape(g, J.dp, &J.sh, code_num_sms(code))) return TSX_EUNSUPPORTED;
    const long long N = p->n_samples;
    J.N = N;
    J.chunk = chunk > 0 && chunk < N ? chunk : N;
    J.n_chunks = N > 0 ? (N + J.chunk - 1) / J.chunk : 0;

    // sigma^2 = 1 / (2 R Eb/N0); float constants and log-weight coefficients
    const double ebn0 = pow(10.0, p->ebn0_db / 10.0);
    const double s2 = 1.0 / (2.0 * rate * ebn0);
    IsArgs &ia = J.ia;
    ia.job = p->job_key;
    ia.s0 = (unsigned long long)p->sample_begin;
    ia.nsamp = N;
    ia.sigf = (float)sqrt(s2);
    ia.muf = (float)p->mu;
    ia.cq = (float)(16.0 / s2);
    ia.A = p->mu / s2;
    ia.Bc = p->mu * p->mu / (2.0 * s2);
    J.Ts.assign(ts_vars, ts_vars + a);
    std::sort(J.Ts.begin(), J.Ts.end());
    J.Ts.erase(std::unique(J.Ts.begin(), J.Ts.end()), J.Ts.end());
    ia.a = (int)J.Ts.size();

    // one device block: T | fail*w | fail | log w | partial sums | sums | counters | queues
    J.nb = (int)((N + kRedChunk - 1) / kRedChunk);
    auto r256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t off_w = 256 + r256((size_t)ia.a * 4);
    const size_t off_f = off_w + r256((size_t)N * 8);
    const size_t off_l = off_f + r256((size_t)N);
    J.off_p = off_l + r256((size_t)N * 8);
    J.off_o = J.off_p + r256((size_t)J.nb * 16);
    const size_t off_c = J.off_o + 256;
    J.off_q = off_c + r256(sizeof(Counters));
    J.total = J.off_q + r256((size_t)std::max<long long>(1, J.n_chunks) * 8);
    return TSX_OK;
}

int is_job_bytes(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p, long long chunk,
                 long long *bytes) {
    IsJob J;
    const int st = is_plan(code, ts_vars, a, p, chunk, J);
    if (st == TSX_OK) *bytes = (long long)J.total;
    return st;
}

void is_job_delete(IsJob *J) {
    if (!J) return;
    if (J->B) cudaFreeAsync(J->B, J->st);
    if (J->e0) cudaEventDestroy(J->e0);
    if (J->e1) cudaEventDestroy(J->e1);
    delete J;
}

// Allocates the job's device block and enqueues the sampling launches (one
// per chunk of samples), the fixed-order reduction and the end event.
int is_job_start(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p, cudaStream_t s,
                 long long chunk, int grid_sms, IsJob **out) {
    *out = nullptr;
    IsJob *J = new IsJob();
    int st = is_plan(code, ts_vars, a, p, chunk, *J);
    if (st != TSX_OK) { delete J; return st; }
    J->st = s;
    J->grid_sms = grid_sms > 0 ? std::min(grid_sms, code_num_sms(code)) : code_num_sms(code);
    J->sh.num_sms = J->grid_sms;
    void *blk = nullptr;
    if (cudaMallocAsync(&blk, J->total, s) != cudaSuccess) {
        cudaGetLastError();
        delete J;
        return TSX_ENOMEM;
    }
    J->B = (unsigned char *)blk;
    IsArgs &ia = J->ia;
    ia.T = (const int *)J->B;
    const size_t off_w = 256 + (((size_t)ia.a * 4 + 255) / 256 * 256);
    ia.wfail = (double *)(J->B + off_w);
    ia.fail_out = (unsigned char *)(J->B + off_w + ((size_t)J->N * 8 + 255) / 256 * 256);
    ia.logw_out = (double *)((unsigned char *)ia.fail_out + ((size_t)J->N + 255) / 256 * 256);
    ia.ctr = (Counters *)(J->B + J->off_o + 256);
    unsigned long long *queues = (unsigned long long *)(J->B + J->off_q);
    auto bail = [&](int code_) { is_job_delete(J); return code_; };
    if (cudaEventCreate(&J->e0) != cudaSuccess || cudaEventCreate(&J->e1) != cudaSuccess) return bail(TSX_ECUDA);
    if (ia.a > 0 &&
        cudaMemcpyAsync((void *)ia.T, J->Ts.data(), sizeof(int) * ia.a, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail(TSX_ECUDA);
    if (cudaMemsetAsync(ia.ctr, 0, sizeof(Counters), s) != cudaSuccess ||
        cudaMemsetAsync(queues, 0, 8 * (size_t)std::max<long long>(1, J->n_chunks), s) != cudaSuccess ||
        cudaEventRecord(J->e0, s) != cudaSuccess)
        return bail(TSX_ECUDA);
    const DevCode &g = J->g;
    const bool qc = g.kind == TSX_CODE_QC;
    const bool reg6 = g.dc_min == 6 && g.dc_max == 6;
    for (long long k = 0; k < J->n_chunks; k++) {
        IsArgs ik = ia;
        const long long b0 = k * J->chunk;
        ik.s0 = ia.s0 + (unsigned long long)b0;
        ik.nsamp = std::min<long long>(J->chunk, J->N - b0);
        ik.wfail = ia.wfail + b0;
        ik.fail_out = ia.fail_out + b0;
        ik.logw_out = ia.logw_out + b0;
        ik.queue = queues + k;
        const LaunchShape &sh = J->sh;
        cudaError_t e;
        if (reg6)
            e = qc ? launch_persistent(is_kernel<true, 6, true>, sh, s, g, J->dp, ik, sh.lay, sh.G)
                   : launch_persistent(is_kernel<false, 6, true>, sh, s, g, J->dp, ik, sh.lay, sh.G);
        else if (g.dc_max <= 8)
            e = qc ? launch_persistent(is_kernel<true, 8, false>, sh, s, g, J->dp, ik, sh.lay, sh.G)
                   : launch_persistent(is_kernel<false, 8, false>, sh, s, g, J->dp, ik, sh.lay, sh.G);
        else
            e = qc ? launch_persistent(is_kernel<true, 32, false>, sh, s, g, J->dp, ik, sh.lay, sh.G)
                   : launch_persistent(is_kernel<false, 32, false>, sh, s, g, J->dp, ik, sh.lay, sh.G);
        if (e != cudaSuccess) return bail(TSX_ECUDA);
    }
    if (J->N > 0) {
        reduce_kernel<<<J->nb, kRedBlock, 0, s>>>(ia.wfail, J->N, (double *)(J->B + J->off_p));
        finish_kernel<<<1, 32, 0, s>>>((const double *)(J->B + J->off_p), J->nb, (double *)(J->B + J->off_o));
        if (cudaGetLastError() != cudaSuccess) return bail(TSX_ECUDA);
    }
    if (cudaEventRecord(J->e1, s) != cudaSuccess) return bail(TSX_ECUDA);
    *out = J;
    return TSX_OK;
}

// After the job's stream has passed its end event: results to the host; the
// device block is given back (stream-ordered).
int is_job_finish(IsJob *J, tsx_is_result *out, uint8_t *fail_out, double *logw_out) {
    memset(out, 0, sizeof(*out));
    out->n_samples = J->N;
    if (J->N == 0) return TSX_OK;
    double sums[2] = {0.0, 0.0};
    Counters c{};
    if (cudaEventSynchronize(J->e1) != cudaSuccess ||
        cudaMemcpy(sums, J->B + J->off_o, sizeof(sums), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&c, J->ia.ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (fail_out && cudaMemcpy(fail_out, J->ia.fail_out, J->N, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (logw_out && cudaMemcpy(logw_out, J->ia.logw_out, J->N * 8, cudaMemcpyDeviceToHost) != cudaSuccess))
        return TSX_ECUDA;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, J->e0, J->e1);
    const double N = (double)J->N;
    out->sum_w = sums[0];
    out->sum_w2 = sums[1];
    out->fer = sums[0] / N;
    out->var = (sums[1] / N - out->fer * out->fer) / N;
    out->n_fail = (int64_t)c.n_fail;
    out->decodes = (int64_t)c.decodes;
    out->iterations = (int64_t)c.iterations;
    out->edge_updates = (int64_t)c.edge_updates;
    out->ms = ms;
    cudaFreeAsync(J->B, J->st);
    J->B = nullptr;
    return TSX_OK;
}

}  // namespace tsx

extern "C" int is_fer_estimate(tsx_code *code, const int32_t *ts_vars, int32_t a, const tsx_is_params *p,
                               void *stream, tsx_is_result *out, uint8_t *fail_out, double *logw_out) {
    if (!code || !p || !out) return TSX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    IsJob *J = nullptr;
    int st = is_job_start(code, ts_vars, a, p, s, 0, 0, &J);
    if (st != TSX_OK) return st;
    st = is_job_finish(J, out, fail_out, logw_out);
    is_job_delete(J);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == TSX_OK) st = TSX_ECUDA;
    return st;
}

// The generalized union bound: one importance-sampling job per set, all
// enqueued on the stream before the first is waited for.
extern "C" int union_bound_fer(tsx_code *code, int64_t n_sets, const int32_t *ts_vars, const int64_t *ts_off,
                               const double *mult, const tsx_is_params *params, void *stream, tsx_union_result *out,
                               double *fer_out) {
    if (!code || !params || !out || n_sets < 0) return TSX_EINVAL;
    if (n_sets > 0 && (!ts_vars || !ts_off || !mult)) return TSX_EINVAL;
    memset(out, 0, sizeof(*out));
    for (int64_t i = 0; i < n_sets; i++)
        if (ts_off[i + 1] < ts_off[i] || ts_off[i + 1] - ts_off[i] > code_dev(code)->n) return TSX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return TSX_ECUDA;
    }
    std::vector<IsJob *> jobs;
    int st = TSX_OK;
    for (int64_t i = 0; i < n_sets && st == TSX_OK; i++) {
        tsx_is_params p = *params;
        p.job_key = params->job_key + (uint64_t)i;
        IsJob *J = nullptr;
        st = is_job_start(code, ts_vars + ts_off[i], (int32_t)(ts_off[i + 1] - ts_off[i]), &p, s, 0, 0, &J);
        if (st == TSX_OK) jobs.push_back(J);
    }
    if (st == TSX_OK && cudaEventRecord(e1, s) != cudaSuccess) st = TSX_ECUDA;
    for (size_t i = 0; i < jobs.size(); i++) {
        tsx_is_result r;
        if (st == TSX_OK) {
            st = is_job_finish(jobs[i], &r, nullptr, nullptr);
            if (st == TSX_OK) {
                out->fer_ub += mult[i] * r.fer;
                out->var_ub += mult[i] * mult[i] * r.var;
                out->samples += r.n_samples;
                out->n_fail += r.n_fail;
                out->edge_updates += r.edge_updates;
                if (fer_out) fer_out[i] = r.fer;
            }
        }
        is_job_delete(jobs[i]);
    }
    out->n_sets = (int64_t)jobs.size();
    if (cudaStreamSynchronize(s) != cudaSuccess && st == TSX_OK) st = TSX_ECUDA;
    float ms = 0.0f;
    if (st == TSX_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) out->ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
