// lnms.cu -- the simulation decoder of Sec. III (the FER curves of Fig. 2):
// quantized normalized layered min-sum with LLR, check-to-variable and
// variable-to-check widths of 4, 4 and 6 bits and 20 iterations, and the
// frame-error simulation around it.
//
// Readings (the paper names the widths and nothing else): every quantity is
// a signed integer and a w-bit value saturates to +-(2^(w-1) - 1); a layer
// is a row block of the QC base matrix (its checks touch distinct variable
// nodes, so they are updated in parallel); the posterior P_v starts at the
// saturated channel value and is kept at the variable-to-check width; per
// layer and check, q = sat_v2c(P_v - r) for its edges, then
// r = sign * sat_c2v((alpha_num * m) >> alpha_shift) with m the minimum |q|
// of the other edges (sgn 0 = +1), then P_v = sat_v2c(q + r); after each
// full iteration x = [P < 0] and the syndrome is checked (also before the
// first).  Failure: x != 0 at the end.
//
// One group of G warps owns one frame: P (int8, n) and r (int8, E) in
// shared memory; lanes take the rows of a layer, a barrier separates the
// layers.  Frames come from a work queue: either the caller's LLRs or BPSK
// over AWGN drawn on the device (the noise generator of the
// importance-sampling kernel, mu = 0), the channel LLR 2 y / sigma^2 scaled,
// rounded half away from zero and saturated to the LLR width.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "decode_impl.cuh"
#include "noise.cuh"

namespace tsx {
namespace {

struct LnmsArgs {
    int K, lim_llr, lim_c2v, lim_v2c, an, as;
    const int8_t *llr;           // [n_frames][n] channel values, or null: drawn noise
    unsigned long long job;      // noise: Philox key
    long long f0;                // noise: sample index of frame 0
    float sigf, cq;              // noise: sigma and the LLR scale 2 llr_scale / sigma^2
    long long n_frames;
    unsigned char *fail;         // [n_frames]
    int *iters;                  // [n_frames] or null
    int *weight;                 // [n_frames] or null: Hamming weight of x (bit errors)
    unsigned char *x_out;        // [n_frames][n] or null
    unsigned long long *queue;   // work queue (frames)
    Counters *ctr;
};

struct LnmsLayout {
    int tables_bytes, p_off, r_off, misc_off, slot_bytes;
};

LnmsLayout lnms_layout(const DevCode &g) {
    LnmsLayout L{};
    L.tables_bytes = al16(tab_offsets(g, false).total);
    int x = 0;
    L.p_off = x; x += al16(g.n);
    L.r_off = x; x += al16(g.E);
    L.misc_off = x; x += al16((int)sizeof(Misc));
    L.slot_bytes = x;
    return L;
}

__device__ __forceinline__ int satw(int x, int lim) { return min(max(x, -lim), lim); }

// round half away from zero (exact), clamped before the conversion
__device__ __forceinline__ int round_half_away(float x, int lim) {
    return (int)fminf(fmaxf(roundf(x), (float)-lim), (float)lim);
}

template <int DCMAX>
__global__ void __launch_bounds__(512, 1) lnms_kernel(DevCode g, LnmsArgs a, LnmsLayout lay, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem);
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
    int8_t *P = (int8_t *)(slot + lay.p_off);
    int8_t *R = (int8_t *)(slot + lay.r_off);
    const int n = g.n, Z = g.Z;
    long long my_frames = 0, my_it = 0, my_fail = 0;

    // unsatisfied checks of x = [P < 0] (group total)
    auto unsat = [&]() {
        int u = 0;
        for (int c = gp.gt; c < g.m; c += gp.T) {
            const int i = c / Z, r = c - i * Z;
            const int deg = sg.rdeg[i];
            int par = 0;
            for (int p = 0; p < deg; p++) par ^= P[sg.rjz[i * g.dc_max + p] + wrapZ(r + sg.rs[i * g.dc_max + p], Z)] < 0;
            u += par;
        }
        return gp.sum(u);
    };

    while (true) {
        if (gp.gt == 0) misc->bcast[0] = (long long)atomicAdd(a.queue, 1ull);
        gp.sync();
        const long long f = misc->bcast[0];
        gp.sync();
        if (f >= a.n_frames) break;
        // the channel
        if (a.llr) {
            const int8_t *src = a.llr + f * (long long)n;
            for (int v = gp.gt; v < n; v += gp.T) P[v] = (int8_t)satw(src[v], a.lim_llr);
        } else {
            for (int q = gp.gt; 4 * q < n; q += gp.T) {
                float gq[4];
                normals4(a.job, (unsigned long long)(a.f0 + f), (uint32_t)q, gq);
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int v = 4 * q + j;
                    if (v < n) {
                        const float y = hadd(1.0f, hmul(a.sigf, gq[j]));
                        P[v] = (int8_t)round_half_away(hmul(y, a.cq), a.lim_llr);
                    }
                }
            }
        }
        for (int e = gp.gt; e < g.E; e += gp.T) R[e] = 0;
        gp.sync();
        int u = unsat();
        int k = 0;
        while (u != 0 && k < a.K) {
            k++;
            for (int i = 0; i < g.m_b; i++) {
                const int deg = sg.rdeg[i];
                const int e0 = sg.reoff[i];
                const int32_t *rjz = sg.rjz + i * g.dc_max;
                const int16_t *rs = sg.rs + i * g.dc_max;
                for (int r = gp.gt; r < Z; r += gp.T) {
                    int q[DCMAX], vv[DCMAX];
                    int m1 = 1 << 20, m2 = 1 << 20, neg = 0;
#pragma unroll
                    for (int p = 0; p < DCMAX; p++) {
                        if (p < deg) {
                            const int v = rjz[p] + wrapZ(r + rs[p], Z);
                            vv[p] = v;
                            const int qq = satw((int)P[v] - (int)R[e0 + p * Z + r], a.lim_v2c);
                            q[p] = qq;
                            neg ^= qq < 0;
                            const int mag = abs(qq);
                            m2 = min(m2, max(m1, mag));  // the two smallest magnitudes, no branch
                            m1 = min(m1, mag);
                        }
                    }
#pragma unroll
                    for (int p = 0; p < DCMAX; p++) {
                        if (p < deg) {
                            // the smallest of the others: m2 for an edge at the minimum (with a tie m2 = m1)
                            const int mn = abs(q[p]) == m1 ? m2 : m1;
                            int mag = deg == 1 ? a.lim_c2v : satw((a.an * mn) >> a.as, a.lim_c2v);
                            const int rr = (neg ^ (q[p] < 0)) ? -mag : mag;
                            R[e0 + p * Z + r] = (int8_t)rr;
                            P[vv[p]] = (int8_t)satw(q[p] + rr, a.lim_v2c);
                        }
                    }
                }
                gp.sync();
            }
            u = unsat();
        }
        // x = [P < 0]
        int w = 0;
        for (int v = gp.gt; v < n; v += gp.T) {
            const int bit = P[v] < 0;
            w += bit;
            if (a.x_out) a.x_out[f * (long long)n + v] = (unsigned char)bit;
        }
        w = gp.sum(w);
        if (gp.gt == 0) {
            a.fail[f] = w != 0;
            if (a.iters) a.iters[f] = k;
            if (a.weight) a.weight[f] = w;
        }
        my_frames++;
        my_it += k;
        my_fail += w != 0;
        gp.sync();
    }
    if (gp.gt == 0) {
        atomicAdd(&a.ctr->decodes, (unsigned long long)my_frames);
        atomicAdd(&a.ctr->iterations, (unsigned long long)my_it);
        atomicAdd(&a.ctr->edge_updates, (unsigned long long)my_it * (unsigned long long)g.E);
        atomicAdd(&a.ctr->n_fail, (unsigned long long)my_fail);
    }
}

constexpr int kSmemCta = 226 * 1024;

struct LnmsShape {
    LnmsLayout lay;
    int G, groups, smem;
};

bool lnms_shape(const DevCode &g, LnmsShape *sh) {
    sh->lay = lnms_layout(g);
    const int fit = (kSmemCta - sh->lay.tables_bytes) / sh->lay.slot_bytes;
    if (fit < 1) return false;
    int G = g.Z / 128;
    if (G < 1) G = 1;
    if (G > 4) G = 4;
    int groups = 16 / G;
    if (groups > fit) groups = fit;
    if (G > 1 && groups > 15) groups = 15;
    sh->G = G;
    sh->groups = groups;
    sh->smem = sh->lay.tables_bytes + groups * sh->lay.slot_bytes;
    return true;
}

template <class Kern>
cudaError_t launch_lnms_t(Kern k, const LnmsShape &sh, int num_sms, cudaStream_t st, const DevCode &g,
                          const LnmsArgs &a) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem);
    if (e != cudaSuccess) return e;
    const int threads = sh.groups * sh.G * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, sh.smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k<<<occ * num_sms, threads, sh.smem, st>>>(g, a, sh.lay, sh.G);
    return cudaGetLastError();
}

cudaError_t launch_lnms(const DevCode &g, const LnmsArgs &a, int num_sms, cudaStream_t st) {
    LnmsShape sh;
    if (!lnms_shape(g, &sh)) return cudaErrorInvalidConfiguration;
    if (g.dc_max <= 8) return launch_lnms_t(lnms_kernel<8>, sh, num_sms, st, g, a);
    return launch_lnms_t(lnms_kernel<32>, sh, num_sms, st, g, a);
}

int lnms_check(const tsx_code *code, const tsx_lnms_params *p) {
    if (!code || !p) return TSX_EINVAL;
    if (p->K < 0 || p->K > 100000) return TSX_EINVAL;
    if (p->llr_bits < 2 || p->llr_bits > 8 || p->c2v_bits < 2 || p->c2v_bits > 8 || p->v2c_bits < 2 ||
        p->v2c_bits > 8)
        return TSX_EINVAL;
    if (p->alpha_shift < 0 || p->alpha_shift > 15 || p->alpha_num < 1 || p->alpha_num > (1 << p->alpha_shift))
        return TSX_EINVAL;
    const DevCode &g = *code_dev(code);
    if (g.kind != TSX_CODE_QC) return TSX_EUNSUPPORTED;  // layers are the row blocks of a QC base
    // every row block is one circulant per column block (distinct variable nodes per layer)
    LnmsShape sh;
    if (!lnms_shape(g, &sh)) return TSX_EUNSUPPORTED;
    return TSX_OK;
}

void fill_args(const tsx_lnms_params *p, LnmsArgs &a) {
    a.K = p->K;
    a.lim_llr = (1 << (p->llr_bits - 1)) - 1;
    a.lim_c2v = (1 << (p->c2v_bits - 1)) - 1;
    a.lim_v2c = (1 << (p->v2c_bits - 1)) - 1;
    a.an = p->alpha_num;
    a.as = p->alpha_shift;
}

}  // namespace
}  // namespace tsx

using namespace tsx;

extern "C" void lnms_params_default(tsx_lnms_params *p) {
    if (!p) return;
    p->K = 20;
    p->llr_bits = 4;
    p->c2v_bits = 4;
    p->v2c_bits = 6;
    p->alpha_num = 3;
    p->alpha_shift = 2;
}

extern "C" void sim_params_default(tsx_sim_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->ebn0_db = 4.0;
    p->rate = 0.0;
    p->llr_scale = 1.0;
    p->max_frames = 100000;
    p->max_errors = 200;
    p->job_key = 0;
    p->frame_begin = 0;
}

extern "C" int lnms_decode(tsx_code *code, const tsx_lnms_params *p, const int8_t *llr, int64_t n_frames,
                           uint8_t *fail, int32_t *iters, uint8_t *x, void *stream) {
    int st = lnms_check(code, p);
    if (st != TSX_OK) return st;
    if (n_frames < 0) return TSX_EINVAL;
    if (n_frames == 0) return TSX_OK;
    if (!llr || !fail) return TSX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    Counters *ctr = nullptr;
    if (cudaMallocAsync(&ctr, sizeof(Counters), s) != cudaSuccess) return TSX_ENOMEM;
    LnmsArgs a{};
    fill_args(p, a);
    a.llr = llr;
    a.n_frames = n_frames;
    a.fail = fail;
    a.iters = iters;
    a.x_out = x;
    a.ctr = ctr;
    a.queue = &ctr->next_cand;
    if (cudaMemsetAsync(ctr, 0, sizeof(Counters), s) != cudaSuccess ||
        launch_lnms(*code_dev(code), a, code_num_sms(code), s) != cudaSuccess)
        st = TSX_ECUDA;
    cudaFreeAsync(ctr, s);
    return st;
}

extern "C" int lnms_simulate(tsx_code *code, const tsx_lnms_params *p, const tsx_sim_params *sp, void *stream,
                             tsx_sim_result *out, uint8_t *fail_out) {
    int st = lnms_check(code, p);
    if (st != TSX_OK) return st;
    if (!sp || !out || sp->max_frames < 0 || sp->max_errors < 0 || sp->frame_begin < 0 || !(sp->llr_scale > 0.0))
        return TSX_EINVAL;
    memset(out, 0, sizeof(*out));
    const DevCode &g = *code_dev(code);
    const double R = sp->rate > 0.0 ? sp->rate : 1.0 - (double)g.m / g.n;
    if (!(R > 0.0)) return TSX_EINVAL;
    const double s2 = 1.0 / (2.0 * R * std::pow(10.0, sp->ebn0_db / 10.0));
    cudaStream_t s = (cudaStream_t)stream;
    const long long chunk = 1 << 16;
    unsigned char *d_fail = nullptr;
    int *d_w = nullptr, *d_it = nullptr;
    Counters *ctr = nullptr;
    if (cudaMalloc(&d_fail, chunk) != cudaSuccess) return TSX_ENOMEM;
    if (cudaMalloc(&d_w, sizeof(int) * chunk) != cudaSuccess || cudaMalloc(&d_it, sizeof(int) * chunk) != cudaSuccess ||
        cudaMalloc(&ctr, sizeof(Counters)) != cudaSuccess) {
        cudaFree(d_fail);
        cudaFree(d_w);
        cudaFree(d_it);
        return TSX_ENOMEM;
    }
    std::vector<unsigned char> hf(chunk);
    std::vector<int> hw(chunk), hit(chunk);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms_total = 0.0f;
    LnmsArgs a{};
    fill_args(p, a);
    a.job = sp->job_key;
    a.sigf = (float)std::sqrt(s2);
    a.cq = (float)(2.0 * sp->llr_scale / s2);
    a.fail = d_fail;
    a.weight = d_w;
    a.iters = d_it;
    a.ctr = ctr;
    a.queue = &ctr->next_cand;
    long long done = 0;
    bool stop = false;
    while (!stop && done < sp->max_frames) {
        const long long nf = std::min<long long>(chunk, sp->max_frames - done);
        a.f0 = sp->frame_begin + done;
        a.n_frames = nf;
        float ms = 0.0f;
        if (cudaMemsetAsync(ctr, 0, sizeof(Counters), s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
            launch_lnms(g, a, code_num_sms(code), s) != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
            cudaMemcpyAsync(hf.data(), d_fail, nf, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hw.data(), d_w, sizeof(int) * nf, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hit.data(), d_it, sizeof(int) * nf, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = TSX_ECUDA;
            break;
        }
        ms_total += ms;
        // frames in order up to the one that reaches max_errors
        for (long long i = 0; i < nf; i++) {
            out->frames++;
            out->iterations += hit[i];
            out->edge_updates += (int64_t)hit[i] * g.E;
            if (fail_out) fail_out[done + i] = hf[i];
            if (hf[i]) {
                out->frame_errors++;
                out->bit_errors += hw[i];
                if (sp->max_errors > 0 && out->frame_errors >= sp->max_errors) {
                    stop = true;
                    break;
                }
            }
        }
        done += nf;
    }
    out->ms = ms_total;
    if (out->frames) {
        out->fer = (double)out->frame_errors / out->frames;
        out->ber = (double)out->bit_errors / ((double)out->frames * g.n);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_fail);
    cudaFree(d_w);
    cudaFree(d_it);
    cudaFree(ctr);
    return st;
}
