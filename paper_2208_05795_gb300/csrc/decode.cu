// decode.cu -- host side of the decoding kernel: shared-memory layout,
// launch shape, dispatch to the per-decoder instantiations, and the
// compaction of the trapping-set hash table.
#include "decode_impl.cuh"

namespace tsx {

cudaError_t launch_enum_i16(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, cudaStream_t);
cudaError_t launch_enum_i8(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, cudaStream_t);
cudaError_t launch_enum_spa(const DevCode &, const DecodeParams &, const EnumBuffers &, const LaunchShape &, cudaStream_t);

// ---------------------------------------------------------------------------
// host side: layout, shape, dispatch
// ---------------------------------------------------------------------------
static int msg_bytes(int decoder) { return decoder == TSX_DEC_NMS_I8 ? 1 : (decoder == TSX_DEC_SPA_F32 ? 4 : 2); }
static int post_bytes(int decoder) { return decoder == TSX_DEC_SPA_F32 ? 4 : 2; }

static SlotLayout make_layout(const DevCode &g, int decoder) {
    SlotLayout L{};
    L.tables_bytes = al16(tab_offsets(g).total);
    int rbytes = g.E * msg_bytes(decoder);
    if (rbytes < 4 * g.m) rbytes = 4 * g.m;
    if (rbytes < 2 * g.n) rbytes = 2 * g.n;
    const int nw = (g.n + 31) / 32;
    int x = 0;
    L.r_off = x; x += al16(rbytes);
    L.p_off = x; x += al16(g.n * post_bytes(decoder));
    L.xa_off = x; x += al16(nw * 4);
    L.xb_off = x; x += al16(nw * 4);
    L.misc_off = x; x += al16((int)sizeof(Misc));
    L.slot_bytes = x;
    return L;
}

constexpr int kSmemCta = 227 * 1024;

bool plan_shape(const DevCode &g, int decoder, int G, int groups, int ctas_per_sm, int num_sms,
                LaunchShape *out) {
    LaunchShape sh{};
    sh.lay = make_layout(g, decoder);
    const int room = kSmemCta - sh.lay.tables_bytes;
    const int fit = room / sh.lay.slot_bytes;
    if (fit < 1) return false;
    if (G <= 0) {
        const int want_warps = 24;
        G = (want_warps + fit - 1) / fit;
        const int work = g.m < g.n ? g.m : g.n;
        int gmax = work / 32;
        if (gmax < 1) gmax = 1;
        if (G > gmax) G = gmax;
        if (G > 16) G = 16;  // one 512-thread CTA per codeword at most
        if (G < 1) G = 1;
    }
    int gmax_cta = 16 / G;  // at most 512 threads per CTA
    if (gmax_cta < 1) gmax_cta = 1;
    if (gmax_cta > fit) gmax_cta = fit;
    if (gmax_cta < 1) return false;
    if (groups <= 0 || groups > gmax_cta) groups = gmax_cta;
    sh.G = G;
    sh.groups = groups;
    sh.smem_bytes = sh.lay.tables_bytes + groups * sh.lay.slot_bytes;
    int per_sm = ctas_per_sm;
    if (per_sm <= 0) {
        const int by_smem = (228 * 1024) / (sh.smem_bytes + 1024);
        const int by_threads = 2048 / (groups * G * 32);
        per_sm = by_smem < by_threads ? by_smem : by_threads;
        if (per_sm > 32) per_sm = 32;
        if (per_sm < 1) per_sm = 1;
    }
    sh.ctas = per_sm * num_sms;
    sh.num_sms = num_sms;
    sh.per_sm_req = ctas_per_sm;
    *out = sh;
    return true;
}

cudaError_t launch_enum(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                        const LaunchShape &sh, cudaStream_t st) {
    switch (dp.decoder) {
        case TSX_DEC_NMS_I16: return launch_enum_i16(g, dp, b, sh, st);
        case TSX_DEC_NMS_I8: return launch_enum_i8(g, dp, b, sh, st);
        default: return launch_enum_spa(g, dp, b, sh, st);
    }
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
    if (e != cudaSuccess || !b.record) return e;
    int rb = (int)((n_rec + 255) / 256);
    if (rb > 4096) rb = 4096;
    if (rb < 1) rb = 1;
    remap_kernel<<<rb, 256, 0, st>>>(b, n_rec, slot_map);
    return cudaGetLastError();
}

}  // namespace tsx
