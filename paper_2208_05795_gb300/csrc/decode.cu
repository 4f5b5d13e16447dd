// decode.cu -- host side of the decoding and sieve kernels: shared-memory
// layouts, launch shapes, dispatch, and the compaction of the trapping-set
// hash table.
#include "decode_impl.cuh"

namespace tsx {

// per-decoder translation units
cudaError_t launch_nms16(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, bool pair,
                         cudaStream_t);
cudaError_t launch_nms16_vn(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &,
                            cudaStream_t);
cudaError_t launch_nms8(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, bool pair,
                        cudaStream_t);
cudaError_t launch_spa(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, cudaStream_t);
cudaError_t launch_sieve_kernel(const DevCode &, const EnumBuffers &, const LaunchShape &, int is_float,
                                cudaStream_t);
cudaError_t launch_batch16(const BatchArgs &, int, bool qc, int dc_max, bool reg6, const LaunchShape &,
                           cudaStream_t);
cudaError_t launch_batch8(const BatchArgs &, int, bool qc, int dc_max, bool reg6, const LaunchShape &,
                          cudaStream_t);

namespace {

enum { kLayScalar = 0, kLayPair = 1, kLaySieve = 2, kLayIs = 3, kLayPairVn = 4 };

int msg_bytes(int decoder) { return decoder == TSX_DEC_NMS_I8 ? 1 : (decoder == TSX_DEC_SPA_F32 ? 4 : 2); }
int post_bytes(int decoder) { return decoder == TSX_DEC_SPA_F32 ? 4 : 2; }

SlotLayout make_layout(const DevCode &g, int decoder, int kind) {
    SlotLayout L{};
    L.tables_bytes = al16(tab_offsets(g, kind == kLayPair || kind == kLayIs || kind == kLayPairVn).total);
    const int nw = (g.n + 31) / 32;
    // message slots: QC edges, or the position-major m x dc_max grid of a CSR code
    const int nmsg = g.kind == TSX_CODE_QC ? g.E : g.m * g.dc_max;
    int x = 0;
    if (kind == kLayScalar) {
        L.r_off = x; x += al16(nmsg * msg_bytes(decoder));
        L.p_off = x; x += al16(g.n * post_bytes(decoder));
        L.xa_off = x; x += al16(nw * 4);
        L.xb_off = x; x += al16(nw * 4);
    } else if (kind == kLayPair) {
        const int rsz = decoder == TSX_DEC_NMS_I8 ? 2 : 4;
        const int xstride = (nw + 3) & ~3;
        L.r_off = x; x += al16(nmsg * rsz);
        L.p_off = x; x += al16(2 * g.n * 4);  // current and accumulating posteriors
        L.xa_off = x; x += al16(4 * xstride * 4);
        L.xb_off = L.xa_off;
    } else if (kind == kLayPairVn) {
        const int xstride = (nw + 3) & ~3;
        L.r_off = x; x += al16(nmsg * 4);
        L.p_off = x; x += al16(g.n * 4);  // one posterior buffer, rebuilt by the variable-node pass
        L.xa_off = x; x += al16(4 * xstride * 4);
        L.xb_off = L.xa_off;
    } else if (kind == kLayIs) {
        L.r_off = x; x += al16(nmsg * 4);
        L.p_off = x; x += al16(3 * g.n * 4);  // two posterior buffers and the channel values
        L.xa_off = x; x += al16(nw * 4);      // bitmask of the trapping set
        L.xb_off = L.xa_off;
    } else {
        int rbytes = 4 * g.m;
        if (rbytes < 2 * g.n) rbytes = 2 * g.n;
        L.r_off = x; x += al16(rbytes);
        L.p_off = x; x += al16(2 * g.n);
        L.xa_off = x; x += al16(nw * 4);
        L.xb_off = L.xa_off;
    }
    L.misc_off = x; x += al16((int)sizeof(Misc));
    L.slot_bytes = x;
    return L;
}

// dynamic shared memory of a CTA: 227 KB less 1 KB for the static part (the
// batch kernel's staged item)
constexpr int kSmemCta = 226 * 1024;

bool plan(const DevCode &g, int decoder, int kind, int G, int groups, int ctas_per_sm, int num_sms,
          LaunchShape *out, int max_warps = 16) {
    LaunchShape sh{};
    sh.lay = make_layout(g, decoder, kind);
    const int room = kSmemCta - sh.lay.tables_bytes;
    const int fit = room / sh.lay.slot_bytes;
    if (fit < 1) return false;
    if (kind == kLaySieve) G = 1;
    if (G <= 0) {
        // as many codeword groups as fit (up to one per warp), the warps shared among them
        G = max_warps / (fit < max_warps ? fit : max_warps);
        int work = g.m < g.n ? g.m : g.n;
        // QC passes run block by block (the variable-node-pass form, and the sampling kernel for
        // check degree > 8, run all blocks at once)
        const bool flat = kind == kLayPairVn || (kind == kLayIs && g.dc_max > 8);
        if (g.kind == TSX_CODE_QC && !flat && g.Z < work) work = g.Z;
        int gmax = work / 32;
        if (gmax < 1) gmax = 1;
        if (G > gmax) G = gmax;
        if (G > 16) G = 16;
        if (G < 1) G = 1;
        if (flat && kind == kLayIs && fit == 1) {
            // one sample pair per CTA: the width (up to max_warps) with the fewest checks per
            // thread, the narrowest of those (the pass ends at the group barrier)
            int best = G, best_rows = (g.m + 32 * G - 1) / (32 * G);
            for (int w = 8; w <= max_warps && w <= gmax; w++) {
                const int rows = (g.m + 32 * w - 1) / (32 * w);
                if (rows < best_rows) {
                    best = w;
                    best_rows = rows;
                }
            }
            G = best;
        }
    }
    int gmax_cta = max_warps / G;  // at most 32 * max_warps threads per CTA
    if (gmax_cta < 1) gmax_cta = 1;
    if (gmax_cta > fit) gmax_cta = fit;
    if (G > 1 && gmax_cta > 15) gmax_cta = 15;  // named barriers 1..15
    if (groups <= 0 || groups > gmax_cta) groups = gmax_cta;
    sh.G = G;
    sh.groups = groups;
    sh.smem_bytes = sh.lay.tables_bytes + groups * sh.lay.slot_bytes;
    sh.num_sms = num_sms;
    sh.per_sm_req = ctas_per_sm;
    sh.ctas = num_sms;
    *out = sh;
    return true;
}

// the launch bound of the two-codeword kernel variant launch_pair picks for g
int pair_warps(const DevCode &g) {
    const bool reg6 = g.dc_min == 6 && g.dc_max == 6;
    return pair_kernel_warps(g.kind == TSX_CODE_QC, reg6 ? 6 : g.dc_max <= 8 ? 8 : 32, reg6);
}

// the two-codeword kernel keeps every biased quantity inside 16 bits
bool pair_ok(const DevCode &g, const DecodeParams &dp) {
    if (dp.decoder == TSX_DEC_SPA_F32) return false;
    const int B = dp.decoder == TSX_DEC_NMS_I8 ? 128 : 1024;
    const long long an_sat = (long long)dp.alpha_num * dp.sat;
    if (an_sat >= 65536) return false;
    const long long rmax = an_sat >> dp.alpha_shift;
    if (rmax > (dp.decoder == TSX_DEC_NMS_I8 ? 127 : B)) return false;
    if ((long long)(g.dv_max + 2) * dp.sat > 0x8000 - B) return false;
    if ((long long)g.dv_max * B > 0x8000 - dp.sat) return false;
    return true;
}

}  // namespace

cudaError_t launch_decode(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, int G, int groups,
                          int ctas_per_sm, int num_sms, int force_scalar, cudaStream_t st) {
    LaunchShape sh;
    // the two-codeword kernel where its bounds hold and its layout fits a CTA
    const bool pair = !force_scalar && pair_ok(g, dp) &&
                      plan(g, dp.decoder, kLayPair, G, groups, ctas_per_sm, num_sms, &sh, pair_warps(g));
    // QC codes of large check degree whose two-buffer layout does not fit: the variable-node-pass form
    if (!pair && !force_scalar && pair_ok(g, dp) && g.kind == TSX_CODE_QC && dp.decoder == TSX_DEC_NMS_I16 &&
        g.dc_max > 8 && plan(g, dp.decoder, kLayPairVn, G, groups, ctas_per_sm, num_sms, &sh, kPairWarps))
        return launch_nms16_vn(g, dp, b, sh, st);
    if (!pair && !plan(g, dp.decoder, kLayScalar, G, groups, ctas_per_sm, num_sms, &sh))
        return cudaErrorInvalidConfiguration;
    switch (dp.decoder) {
        case TSX_DEC_NMS_I16: return launch_nms16(g, dp, b, sh, pair, st);
        case TSX_DEC_NMS_I8: return launch_nms8(g, dp, b, sh, pair, st);
        default: return launch_spa(g, dp, b, sh, st);
    }
}

cudaError_t launch_sieve(const DevCode &g, const EnumBuffers &b, int decoder, int num_sms, cudaStream_t st) {
    LaunchShape sh;
    if (!plan(g, decoder, kLaySieve, 1, 0, 0, num_sms, &sh)) return cudaErrorInvalidConfiguration;
    return launch_sieve_kernel(g, b, sh, decoder == TSX_DEC_SPA_F32 ? 1 : 0, st);
}

// variant bits: 1 = QC, 2 = int8 storage, 4 = all check-regular of degree 6,
// bits 8.. = the largest check degree
bool plan_batch(const DevCode *const *g, const DecodeParams *dp, const EnumBuffers *b, const int *G_req, int n,
                int num_sms, BatchItem *items, LaunchShape *common, int *variant) {
    if (n <= 0) return false;
    const int kind = g[0]->kind, dec = dp[0].decoder;
    bool reg6 = true;
    int dcmax = 1, smem = 0;
    for (int i = 0; i < n; i++) {
        if (g[i]->kind != kind || dp[i].decoder != dec || !pair_ok(*g[i], dp[i])) return false;
        LaunchShape sh;
        int G, groups;
        items[i].scalar = 0;
        if (!plan(*g[i], dec, kLayPair, 1, 1, 0, num_sms, &sh)) {
            items[i].scalar = 1;  // decoded by a launch of its own
            continue;
        }
        reg6 = reg6 && g[i]->dc_min == 6 && g[i]->dc_max == 6;
        if (g[i]->dc_max > dcmax) dcmax = g[i]->dc_max;
        if (G_req && G_req[i] > 0) {
            // the requested (tuned) group width, as many groups as fit
            if (!plan(*g[i], dec, kLayPair, G_req[i], 0, 0, num_sms, &sh)) return false;
            G = sh.G;
            groups = sh.groups;
        } else {
            // the single-code launch's automatic shape
            if (!plan(*g[i], dec, kLayPair, 0, 0, 0, num_sms, &sh)) return false;
            G = sh.G;
            groups = sh.groups;
        }
        items[i].g = *g[i];
        items[i].dp = dp[i];
        items[i].b = b[i];
        items[i].lay = sh.lay;
        items[i].G = G;
        items[i].groups = groups;
        const int need = sh.lay.tables_bytes + groups * sh.lay.slot_bytes;
        if (need > smem) smem = need;
    }
    LaunchShape sh{};
    sh.G = 1;
    sh.groups = 16;
    sh.smem_bytes = smem;
    sh.num_sms = num_sms;
    sh.per_sm_req = 0;
    sh.ctas = num_sms;
    *common = sh;
    *variant = (kind == TSX_CODE_QC ? 1 : 0) | (dec == TSX_DEC_NMS_I8 ? 2 : 0) | (reg6 ? 4 : 0) | (dcmax << 8);
    return true;
}

cudaError_t launch_batch(const BatchArgs &items, int n, int variant, const LaunchShape &sh, cudaStream_t st) {
    const bool qc = variant & 1, i8 = variant & 2, reg6 = variant & 4;
    const int dcmax = variant >> 8;
    return i8 ? launch_batch8(items, n, qc, dcmax, reg6, sh, st) : launch_batch16(items, n, qc, dcmax, reg6, sh, st);
}

bool plan_is_shape(const DevCode &g, const DecodeParams &dp, LaunchShape *sh, int num_sms) {
    if (!pair_ok(g, dp)) return false;
    // the flat form (QC, check degree > 8) is launched with up to kIsWarps warps, the others with 16
    return plan(g, TSX_DEC_NMS_I16, kLayIs, 0, 0, 0, num_sms, sh,
                g.kind == TSX_CODE_QC && g.dc_max > 8 ? kIsWarps : 16);
}

bool decode_fits(const DevCode &g, int decoder) {
    LaunchShape sh;
    return plan(g, decoder, kLayScalar, 1, 1, 0, 1, &sh) && plan(g, decoder, kLaySieve, 1, 1, 0, 1, &sh);
}

// ---------------------------------------------------------------------------
// compaction of the hash table
// ---------------------------------------------------------------------------
__global__ void compact_kernel(EnumBuffers b, int *ts_off, int *ts_count, int *ts_thr, int *slot_map) {
    for (unsigned long long s = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; s <= b.cap_mask;
         s += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long tag = b.tags[s];
        if (!tag) continue;
        const unsigned idx = atomicAdd(&b.ctr->n_ts, 1u);
        ts_off[idx] = (int)(tag & 0xffffffffull);
        ts_count[idx] = b.t_count[s];
        ts_thr[idx] = b.t_thr[s];
        slot_map[s] = (int)idx;
    }
}

__global__ void remap_kernel(EnumBuffers b, long long n_rec, const int *slot_map) {
    const long long total = (long long)b.ctr->n_cand_total;
    const long long end = b.cand_end < 0 || b.cand_end > total ? total : b.cand_end;
    long long n = end - b.cand_begin;
    if (n > n_rec) n = n_rec;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = b.c_slot[i];
        if (s >= 0) b.c_slot[i] = slot_map[s];
    }
}

cudaError_t launch_compact(const EnumBuffers &b, long long n_rec, int *ts_off, int *ts_count, int *ts_thr,
                           int *slot_map, cudaStream_t st) {
    const long long cap = (long long)b.cap_mask + 1;
    int blocks = (int)((cap + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    compact_kernel<<<blocks, 256, 0, st>>>(b, ts_off, ts_count, ts_thr, slot_map);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int rb = (int)((n_rec + 255) / 256);
    if (rb > 4096) rb = 4096;
    if (rb < 1) rb = 1;
    remap_kernel<<<rb, 256, 0, st>>>(b, n_rec, slot_map);
    return cudaGetLastError();
}

}  // namespace tsx
