// api.cu -- the C ABI (include/tsx.h): code loading, the enumeration
// pipeline on a stream, and host views of its results.
//
// Host code here only validates, builds the per-code tables once, sizes
// buffers and orders kernel launches; every step of the enumeration itself
// runs in the kernels of cand.cu and decode.cu.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <deque>
#include <numeric>
#include <vector>

#include "kernels.cuh"

using namespace tsx;

#define CK(x)                                 \
    do {                                      \
        cudaError_t e__ = (x);                \
        if (e__ != cudaSuccess) return TSX_ECUDA; \
    } while (0)

struct tsx_code {
    DevCode d{};
    tsx_code_info info{};
    void *dev = nullptr;  // one allocation for all tables
    std::vector<int64_t> ball_ptr;  // host copy
    int device = 0;
    int num_sms = 0;
    // cycles through each representative: closed walks of 2 and 3 variable
    // nodes (twice the 4- and 6-cycles), and the iteration-budget weight
    // 2 c4(v) + c6(v) of every variable node on the device
    std::vector<int64_t> walks4, walks6;
    int *vweight = nullptr;
};

struct tsx_ts_list {
    tsx_code *code = nullptr;
    cudaStream_t st = nullptr;
    tsx_enum_params p{};
    DecodeParams dp{};
    long long n_rec = 0;  // record capacity
    long long cap = 0;    // hash-table slots
    long long pool_cap = 0;
    std::vector<void *> bufs;
    EnumBuffers b{};
    Counters *ctr = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // start, decode, sieve, compact, end
    int *ts_off = nullptr, *ts_count = nullptr, *ts_thr = nullptr, *slot_map = nullptr;
    // candidate generation
    std::vector<long long> raw_off;
    long long raw_total = 0, n_chunks = 0, paths = 0;
    int cyc_l = 0;
    bool cycles = false, events = true;
    long long *d_raw_off = nullptr, *d_chunk_off = nullptr, *d_cyc_off = nullptr;
    int *d_chunk_cnt = nullptr, *d_cyc_cnt = nullptr;
    // decode launch shape: one launch over the whole range (dchunk = 0) or
    // one launch per dchunk candidates, each with its own queue word
    long long dchunk = 0, n_dchunks = 0, range_end = 0;
    long long cand_bound = 0;
    unsigned long long *d_queues = nullptr;
    int grid_sms = 0;
    // sizing only: allocations are counted, not made
    bool dry = false;
    long long bytes = 0;
    // host results
    bool oom = false;
    bool fetched = false;
    int fetch_status = TSX_OK;
    tsx_enum_stats stats{};
    std::vector<int32_t> a, b_, orbit, count, thr, flags, vars;
    std::vector<float> thr_f;
    std::vector<int64_t> var_off;
    std::vector<int32_t> cvars, cthr, cts, cflags, cdec, cit;
    std::vector<float> cthr_f;
};

extern "C" const char *tsx_strerror(int s) {
    switch (s) {
        case TSX_OK: return "ok";
        case TSX_EINVAL: return "invalid argument";
        case TSX_ENOMEM: return "out of memory or a device table overflowed";
        case TSX_ECUDA: return "CUDA runtime error";
        case TSX_ETIMEDOUT: return "device-side wait timed out";
        case TSX_EBUSY: return "resource busy";
        case TSX_EUNSUPPORTED: return "size or degree above the compiled limits";
        case TSX_ENOTFOUND: return "unknown id";
        case TSX_EAGAIN: return "not finished";
        default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// load_code
// ---------------------------------------------------------------------------
namespace {

struct HostTables {
    int kind, n, m, E, Z = 0, n_b = 0, m_b = 0, dv_max = 1, dc_max = 1;
    std::vector<int16_t> rdeg, rs, cdeg, cs;
    std::vector<int32_t> reoff, rjz, ceoff, ciz;
    std::vector<uint16_t> c_ptr, c_vn, v_ptr, v_edge, v_chk;
    // generic adjacency for the girth search
    std::vector<std::vector<int>> vadj, cadj;
};

int build_qc(const tsx_code_desc &d, HostTables &h) {
    if (d.m_b <= 0 || d.n_b <= 0 || d.Z <= 0 || !d.shifts) return TSX_EINVAL;
    if (d.n_b > TSX_MAX_NB || d.m_b > kMaxMb) return TSX_EUNSUPPORTED;
    if ((long long)d.n_b * d.Z > TSX_MAX_N || (long long)d.m_b * d.Z > 65535) return TSX_EUNSUPPORTED;
    h.kind = TSX_CODE_QC;
    h.Z = d.Z; h.n_b = d.n_b; h.m_b = d.m_b;
    h.n = d.n_b * d.Z; h.m = d.m_b * d.Z;
    std::vector<int> rd(d.m_b, 0), cd(d.n_b, 0);
    for (int i = 0; i < d.m_b; i++)
        for (int j = 0; j < d.n_b; j++) {
            int a = d.shifts[i * d.n_b + j];
            if (a < -1 || a >= d.Z) return TSX_EINVAL;
            if (a >= 0) { rd[i]++; cd[j]++; }
        }
    h.dc_max = std::max(1, *std::max_element(rd.begin(), rd.end()));
    h.dv_max = std::max(1, *std::max_element(cd.begin(), cd.end()));
    if (h.dc_max > TSX_MAX_DC || h.dv_max > TSX_MAX_DV) return TSX_EUNSUPPORTED;
    h.rdeg.assign(d.m_b, 0); h.reoff.assign(d.m_b, 0);
    h.rjz.assign(d.m_b * h.dc_max, 0); h.rs.assign(d.m_b * h.dc_max, 0);
    h.cdeg.assign(d.n_b, 0); h.ceoff.assign(d.n_b * h.dv_max, 0);
    h.cs.assign(d.n_b * h.dv_max, 0); h.ciz.assign(d.n_b * h.dv_max, 0);
    std::vector<int> pos(d.m_b * d.n_b, -1);
    long long e = 0;
    for (int i = 0; i < d.m_b; i++) {
        h.reoff[i] = (int)e;
        int p = 0;
        for (int j = 0; j < d.n_b; j++) {
            int a = d.shifts[i * d.n_b + j];
            if (a < 0) continue;
            h.rjz[i * h.dc_max + p] = j * d.Z;
            h.rs[i * h.dc_max + p] = (int16_t)a;
            pos[i * d.n_b + j] = p++;
        }
        h.rdeg[i] = (int16_t)p;
        e += (long long)p * d.Z;
    }
    if (e > 0x7fffffffLL) return TSX_EUNSUPPORTED;
    h.E = (int)e;
    for (int j = 0; j < d.n_b; j++) {
        int t = 0;
        for (int i = 0; i < d.m_b; i++) {
            int a = d.shifts[i * d.n_b + j];
            if (a < 0) continue;
            h.ceoff[j * h.dv_max + t] = h.reoff[i] + pos[i * d.n_b + j] * d.Z;
            h.cs[j * h.dv_max + t] = (int16_t)a;
            h.ciz[j * h.dv_max + t] = i * d.Z;
            t++;
        }
        h.cdeg[j] = (int16_t)t;
    }
    return TSX_OK;
}

int build_csr(const tsx_code_desc &d, HostTables &h) {
    if (d.n <= 0 || d.m <= 0 || !d.row_ptr || !d.col_idx) return TSX_EINVAL;
    if (d.n > TSX_MAX_N || d.m > 65534) return TSX_EUNSUPPORTED;
    if (d.row_ptr[0] != 0) return TSX_EINVAL;
    for (int c = 0; c < d.m; c++)
        if (d.row_ptr[c + 1] < d.row_ptr[c]) return TSX_EINVAL;
    long long E = d.row_ptr[d.m];
    if (E <= 0) return TSX_EINVAL;
    if (E > 65535) return TSX_EUNSUPPORTED;
    h.kind = TSX_CODE_CSR;
    h.n = d.n; h.m = d.m; h.E = (int)E;
    h.c_ptr.resize(d.m + 1);
    h.c_vn.resize(E);
    std::vector<int> vd(d.n, 0);
    for (int c = 0; c < d.m; c++) {
        std::vector<int> row(d.col_idx + d.row_ptr[c], d.col_idx + d.row_ptr[c + 1]);
        std::sort(row.begin(), row.end());
        for (size_t k = 0; k < row.size(); k++) {
            if (row[k] < 0 || row[k] >= d.n) return TSX_EINVAL;
            if (k && row[k] == row[k - 1]) return TSX_EINVAL;
            h.c_vn[d.row_ptr[c] + k] = (uint16_t)row[k];
            vd[row[k]]++;
        }
        h.c_ptr[c] = (uint16_t)d.row_ptr[c];
        h.dc_max = std::max(h.dc_max, (int)row.size());
    }
    h.c_ptr[d.m] = (uint16_t)E;
    h.dv_max = std::max(1, *std::max_element(vd.begin(), vd.end()));
    if (h.dc_max > TSX_MAX_DC || h.dv_max > TSX_MAX_DV) return TSX_EUNSUPPORTED;
    h.v_ptr.assign(d.n + 1, 0);
    for (int v = 0; v < d.n; v++) h.v_ptr[v + 1] = (uint16_t)(h.v_ptr[v] + vd[v]);
    // messages are stored position-major: edge (c, p) at p*m + c
    if ((long long)h.dc_max * d.m > 65535) return TSX_EUNSUPPORTED;
    h.v_edge.resize(E);
    h.v_chk.resize(E);
    std::vector<int> fill(d.n, 0);
    for (int c = 0; c < d.m; c++)  // checks ascending -> edges of v ascending by check
        for (int e = h.c_ptr[c]; e < h.c_ptr[c + 1]; e++) {
            int v = h.c_vn[e];
            int t = h.v_ptr[v] + fill[v]++;
            h.v_edge[t] = (uint16_t)((e - h.c_ptr[c]) * d.m + c);
            h.v_chk[t] = (uint16_t)c;
        }
    return TSX_OK;
}

void adjacency(HostTables &h) {
    h.vadj.assign(h.n, {});
    h.cadj.assign(h.m, {});
    if (h.kind == TSX_CODE_QC) {
        for (int i = 0; i < h.m_b; i++)
            for (int p = 0; p < h.rdeg[i]; p++) {
                int jz = h.rjz[i * h.dc_max + p], a = h.rs[i * h.dc_max + p];
                for (int r = 0; r < h.Z; r++) {
                    int c = i * h.Z + r, v = jz + (r + a) % h.Z;
                    h.cadj[c].push_back(v);
                    h.vadj[v].push_back(c);
                }
            }
    } else {
        for (int c = 0; c < h.m; c++)
            for (int e = h.c_ptr[c]; e < h.c_ptr[c + 1]; e++) {
                h.cadj[c].push_back(h.c_vn[e]);
                h.vadj[h.c_vn[e]].push_back(c);
            }
    }
}

// Shortest cycle by breadth-first search from each start node (QC: the
// n_b nodes (j,0) suffice by the circulant symmetry).
int girth_of(const HostTables &h) {
    const int N = h.n + h.m;
    std::vector<int> dist(N), par(N), q(N);
    int best = 1 << 30;
    const int starts = h.kind == TSX_CODE_QC ? h.n_b : h.n;
    for (int si = 0; si < starts; si++) {
        int s = h.kind == TSX_CODE_QC ? si * h.Z : si;
        std::fill(dist.begin(), dist.end(), -1);
        int qh = 0, qt = 0;
        dist[s] = 0; par[s] = -1; q[qt++] = s;
        while (qh < qt) {
            int u = q[qh++];
            if (2 * dist[u] + 1 >= best) break;
            const std::vector<int> &nb = u < h.n ? h.vadj[u] : h.cadj[u - h.n];
            for (int x : nb) {
                int w = u < h.n ? h.n + x : x;
                if (w == par[u]) continue;
                if (dist[w] < 0) { dist[w] = dist[u] + 1; par[w] = u; q[qt++] = w; }
                else best = std::min(best, dist[u] + dist[w] + 1);
            }
        }
    }
    return best == (1 << 30) ? 0 : best;
}

template <class T>
size_t put(std::vector<unsigned char> &blob, const std::vector<T> &v) {
    size_t off = (blob.size() + 255) & ~size_t(255);
    blob.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

}  // namespace

extern "C" int load_code(const tsx_code_desc *desc, void *stream, tsx_code **out) {
    if (!desc || !out) return TSX_EINVAL;
    *out = nullptr;
    HostTables h;
    int st = desc->kind == TSX_CODE_QC ? build_qc(*desc, h)
             : desc->kind == TSX_CODE_CSR ? build_csr(*desc, h)
                                          : TSX_EINVAL;
    if (st != TSX_OK) return st;
    if (h.E == 0) return TSX_EINVAL;
    adjacency(h);
    const int girth = girth_of(h);
    h.vadj.clear(); h.cadj.clear();

    tsx_code *c = new tsx_code();
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return TSX_ECUDA;
    }
    std::vector<unsigned char> blob;
    size_t o_rdeg = put(blob, h.rdeg), o_reoff = put(blob, h.reoff), o_rjz = put(blob, h.rjz),
           o_rs = put(blob, h.rs), o_cdeg = put(blob, h.cdeg), o_ceoff = put(blob, h.ceoff),
           o_cs = put(blob, h.cs), o_ciz = put(blob, h.ciz), o_cptr = put(blob, h.c_ptr),
           o_cvn = put(blob, h.c_vn), o_vptr = put(blob, h.v_ptr), o_vedge = put(blob, h.v_edge),
           o_vchk = put(blob, h.v_chk);
    blob.resize((blob.size() + 255) & ~size_t(255));
    const int n_rep = h.kind == TSX_CODE_QC ? h.n_b : h.n;
    size_t o_bptr = blob.size();
    blob.resize(o_bptr + sizeof(int64_t) * (n_rep + 1));
    size_t o_sizes = (blob.size() + 255) & ~size_t(255);
    blob.resize(o_sizes + sizeof(int) * n_rep);
    unsigned char *dev = nullptr;
    if (cudaMalloc(&dev, blob.size()) != cudaSuccess) { delete c; return TSX_ENOMEM; }
    c->dev = dev;
    auto fail = [&](int code) { cudaFree(dev); delete c; return code; };
    if (cudaMemcpyAsync(dev, blob.data(), blob.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return fail(TSX_ECUDA);
    DevCode &d = c->d;
    d.kind = h.kind; d.n = h.n; d.m = h.m; d.E = h.E; d.Z = h.Z; d.n_b = h.n_b; d.m_b = h.m_b;
    d.dv_max = h.dv_max; d.dc_max = h.dc_max; d.girth = girth;
    d.dv_min = h.dv_max;
    if (h.kind == TSX_CODE_QC)
        for (int j = 0; j < h.n_b; j++) d.dv_min = std::min<int>(d.dv_min, h.cdeg[j]);
    else
        for (int v = 0; v < h.n; v++) d.dv_min = std::min<int>(d.dv_min, h.v_ptr[v + 1] - h.v_ptr[v]);
    d.dc_min = h.dc_max;
    for (int c = 0; c < (h.kind == TSX_CODE_QC ? h.m_b : h.m); c++) {
        const int dc = h.kind == TSX_CODE_QC ? h.rdeg[c] : h.c_ptr[c + 1] - h.c_ptr[c];
        if (dc < d.dc_min) d.dc_min = dc;
    }
    d.wstart = std::max(1, girth / 2);
    d.n_rep = n_rep;
    d.rdeg = (const int16_t *)(dev + o_rdeg); d.reoff = (const int32_t *)(dev + o_reoff);
    d.rjz = (const int32_t *)(dev + o_rjz); d.rs = (const int16_t *)(dev + o_rs);
    d.cdeg = (const int16_t *)(dev + o_cdeg); d.ceoff = (const int32_t *)(dev + o_ceoff);
    d.cs = (const int16_t *)(dev + o_cs); d.ciz = (const int32_t *)(dev + o_ciz);
    d.c_ptr = (const uint16_t *)(dev + o_cptr); d.c_vn = (const uint16_t *)(dev + o_cvn);
    d.v_ptr = (const uint16_t *)(dev + o_vptr); d.v_edge = (const uint16_t *)(dev + o_vedge);
    d.v_chk = (const uint16_t *)(dev + o_vchk);
    d.ball_ptr = (const int64_t *)(dev + o_bptr);
    int *sizes = (int *)(dev + o_sizes);
    // Tanner balls: count, prefix on the host, write
    if (launch_ball(d, sizes, nullptr, nullptr, false, s) != cudaSuccess) return fail(TSX_ECUDA);
    std::vector<int> hs(n_rep);
    if (cudaMemcpyAsync(hs.data(), sizes, sizeof(int) * n_rep, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(TSX_ECUDA);
    c->ball_ptr.assign(n_rep + 1, 0);
    for (int r = 0; r < n_rep; r++) c->ball_ptr[r + 1] = c->ball_ptr[r] + hs[r];
    int32_t *ball = nullptr;
    if (cudaMalloc(&ball, sizeof(int32_t) * std::max<int64_t>(1, c->ball_ptr[n_rep])) != cudaSuccess)
        return fail(TSX_ENOMEM);
    d.ball = ball;
    if (cudaMemcpyAsync(dev + o_bptr, c->ball_ptr.data(), sizeof(int64_t) * (n_rep + 1),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        launch_ball(d, sizes, d.ball_ptr, ball, true, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(ball);
        return fail(TSX_ECUDA);
    }
    // 4- and 6-cycles through the representatives (Table V's densities), for the iteration budgets
    {
        unsigned long long *walks = nullptr;
        if (cudaMalloc(&walks, sizeof(unsigned long long) * n_rep * (kCycLmax + 1)) != cudaSuccess) {
            cudaFree(ball);
            return fail(TSX_ENOMEM);
        }
        std::vector<unsigned long long> hw((size_t)n_rep * (kCycLmax + 1));
        if (launch_cycles(d, 3, walks, nullptr, s) != cudaSuccess ||
            cudaMemcpyAsync(hw.data(), walks, sizeof(unsigned long long) * hw.size(), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFree(walks);
            cudaFree(ball);
            return fail(TSX_ECUDA);
        }
        cudaFree(walks);
        c->walks4.resize(n_rep);
        c->walks6.resize(n_rep);
        for (int r = 0; r < n_rep; r++) {
            c->walks4[r] = (int64_t)hw[(size_t)r * (kCycLmax + 1) + 2];
            c->walks6[r] = (int64_t)hw[(size_t)r * (kCycLmax + 1) + 3];
        }
        std::vector<int> vw(h.n);
        for (int v = 0; v < h.n; v++) {
            const int r = h.kind == TSX_CODE_QC ? v / h.Z : v;
            const int64_t w = c->walks4[r] + c->walks6[r] / 2;
            vw[v] = (int)std::min<int64_t>(w, 1 << 28);
        }
        if (cudaMalloc(&c->vweight, sizeof(int) * h.n) != cudaSuccess) {
            cudaFree(ball);
            return fail(TSX_ENOMEM);
        }
        if (cudaMemcpyAsync(c->vweight, vw.data(), sizeof(int) * h.n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaFree(c->vweight);
            cudaFree(ball);
            return fail(TSX_ECUDA);
        }
    }
    tsx_code_info &in = c->info;
    in.kind = h.kind; in.n = h.n; in.m = h.m; in.E = h.E; in.Z = h.Z; in.n_b = h.n_b; in.m_b = h.m_b;
    in.dv_max = h.dv_max; in.dc_max = h.dc_max; in.girth = girth; in.n_rep = n_rep;
    in.ball_total = c->ball_ptr[n_rep];
    in.device_bytes = (int64_t)blob.size() + sizeof(int32_t) * (in.ball_total + h.n);
    *out = c;
    return TSX_OK;
}

extern "C" void free_code(tsx_code *c) {
    if (!c) return;
    cudaFree((void *)c->d.ball);
    cudaFree(c->vweight);
    cudaFree(c->dev);
    delete c;
}

extern "C" int cycle_counts(const tsx_code *c, int64_t *c4, int64_t *c6) {
    if (!c || !c4 || !c6) return TSX_EINVAL;
    const DevCode &d = c->d;
    for (int v = 0; v < d.n; v++) {
        const int r = d.kind == TSX_CODE_QC ? v / d.Z : v;
        c4[v] = c->walks4[r] / 2;
        c6[v] = c->walks6[r] / 2;
    }
    return TSX_OK;
}

extern "C" int emd_spectrum(tsx_code *c, int32_t lmax, void *stream, tsx_emd_spectrum *out) {
    if (!c || !out || lmax < 2 || lmax > kCycLmax) return TSX_EINVAL;
    memset(out, 0, sizeof(*out));
    const DevCode &d = c->d;
    // walk nodes of the search: n_rep dv (dc - 1) ((dv - 1)(dc - 1))^(lmax - 2)
    double work = (double)d.n_rep * d.dv_max * std::max(1, d.dc_max - 1);
    for (int l = 2; l < lmax; l++) work *= (double)std::max(1, d.dv_max - 1) * std::max(1, d.dc_max - 1);
    if (work > 4e11) return TSX_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *buf = nullptr;
    const size_t nw = (size_t)d.n_rep * (kCycLmax + 1), nh = (size_t)(kCycLmax + 1) * kEmdBins;
    if (cudaMalloc(&buf, sizeof(unsigned long long) * (nw + nh)) != cudaSuccess) return TSX_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<unsigned long long> hw(nw), hh(nh);
    int st = TSX_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventRecord(e0, s) != cudaSuccess || launch_cycles(d, lmax, buf, buf + nw, s) != cudaSuccess ||
        cudaEventRecord(e1, s) != cudaSuccess ||
        cudaMemcpyAsync(hw.data(), buf, sizeof(unsigned long long) * nw, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hh.data(), buf + nw, sizeof(unsigned long long) * nh, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        st = TSX_ECUDA;
    if (st == TSX_OK) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        out->ms = ms;
        out->lmax = lmax;
        for (size_t r = 0; r < (size_t)d.n_rep; r++)
            for (int l = 2; l <= lmax; l++) out->walks[l] += (int64_t)hw[r * (kCycLmax + 1) + l];
        for (int l = 2; l <= lmax; l++)
            for (int e = 0; e < kEmdBins; e++) out->count2l[l][e] = (int64_t)hh[(size_t)l * kEmdBins + e];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    return st;
}

extern "C" int code_info(const tsx_code *c, tsx_code_info *info) {
    if (!c || !info) return TSX_EINVAL;
    *info = c->info;
    return TSX_OK;
}

// ---------------------------------------------------------------------------
// enumerate_ts
// ---------------------------------------------------------------------------
extern "C" void enum_params_default(tsx_enum_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->decoder = TSX_DEC_NMS_I16;
    p->K = 20;
    p->base_llr = 16;
    p->sat = 511;
    p->alpha_num = 3;
    p->alpha_shift = 2;
    p->amp_steps = 10;
    p->spa_clip = 30.0f;
    p->spa_amax = 64.0f;
    p->max_size = 3;
    p->cycle_len = 0;
    p->record_candidates = 1;
    p->cand_begin = 0;
    p->cand_end = -1;
}

static int check_params(const tsx_enum_params &p) {
    if (p.decoder < 0 || p.decoder > 2) return TSX_EINVAL;
    if (p.K < 0 || p.K > 100000) return TSX_EINVAL;
    if (p.base_llr <= 0) return TSX_EINVAL;
    if (p.decoder != TSX_DEC_SPA_F32) {
        if (p.sat < 1 || p.sat > 8191) return TSX_EINVAL;
        if (p.decoder == TSX_DEC_NMS_I8 && p.sat > 169) return TSX_EUNSUPPORTED;
        if (p.alpha_shift < 0 || p.alpha_shift > 15) return TSX_EINVAL;
        if (p.alpha_num < 1 || p.alpha_num > (1 << p.alpha_shift)) return TSX_EINVAL;
        if (p.amp_steps < 1 || p.amp_steps > 20) return TSX_EINVAL;
    } else {
        if (!(p.spa_clip > 0.0f) || !(p.spa_amax > 0.0f)) return TSX_EINVAL;
        if (p.amp_steps < 0 || p.amp_steps > 24) return TSX_EINVAL;
    }
    if (p.max_size < 1 || p.max_size > 4) return TSX_EINVAL;
    if (p.cycle_len != 0 && (p.cycle_len < 4 || p.cycle_len > 8 || (p.cycle_len & 1))) return TSX_EINVAL;
    if (p.cand_begin < 0) return TSX_EINVAL;
    if (p.cand_end >= 0 && p.cand_end < p.cand_begin) return TSX_EINVAL;
    if (p.warps_per_cta < 0 || p.warps_per_cta > 16 || p.ctas_per_sm < 0) return TSX_EINVAL;
    if (p.kernel < 0 || p.kernel > 2) return TSX_EINVAL;
    if (p.list_mode < 0 || p.list_mode > 1 || p.kstart < -1) return TSX_EINVAL;
    if (p.list_mode && p.decoder == TSX_DEC_SPA_F32) return TSX_EUNSUPPORTED;
    if (p.list_mode && p.K > 1000) return TSX_EUNSUPPORTED;
    if (p.budget_wref < 0) return TSX_EINVAL;
    if (p.budget_wref > 0 && (p.budget_kmin < 1 || p.budget_kmin > p.K || p.K > 65535)) return TSX_EINVAL;
    return TSX_OK;
}

// accessors for the other translation units of the library
namespace tsx {
const DevCode *code_dev(const tsx_code *c) { return &c->d; }
int code_num_sms(const tsx_code *c) { return c->num_sms; }
int code_device(const tsx_code *c) { return c->device; }
int enum_params_to_decode(const tsx_enum_params *p, DecodeParams *dp) {
    const int st = check_params(*p);
    if (st != TSX_OK) return st;
    dp->decoder = p->decoder; dp->K = p->K; dp->base_llr = p->base_llr; dp->sat = p->sat;
    dp->alpha_num = p->alpha_num; dp->alpha_shift = p->alpha_shift; dp->amp_steps = p->amp_steps;
    dp->spa_clip = p->spa_clip; dp->spa_amax = p->spa_amax;
    return TSX_OK;
}
}  // namespace tsx

static long long next_pow2(long long x) {
    long long p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <class T>
static T *lalloc(tsx_ts_list *L, size_t count, cudaStream_t s) {
    const size_t bytes = std::max<size_t>(1, count) * sizeof(T);
    L->bytes += (long long)((bytes + 255) / 256 * 256);
    if (L->dry) return nullptr;
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        L->oom = true;
        return nullptr;
    }
    L->bufs.push_back(p);
    return (T *)p;
}

static void release(tsx_ts_list *L) {
    for (void *p : L->bufs) cudaFreeAsync(p, L->st);
    L->bufs.clear();
    for (cudaEvent_t &e : L->ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
}

// Validates, sizes and allocates the buffers of one enumeration (no kernel
// is launched; the raw-set offsets are uploaded).
// With dry = true nothing is allocated or copied: *out receives a list whose
// `bytes` is the device memory the real call would take (free it with
// delete).  dchunk > 0 splits the decode into launches of dchunk candidates;
// grid_sms > 0 caps the decode and sieve grids at that many SMs.
static int prepare_list(tsx_code *code, const tsx_enum_params *params, cudaStream_t s, bool events,
                        tsx_ts_list **out, long long dchunk = 0, int grid_sms = 0, bool dry = false) {
    *out = nullptr;
    int st = check_params(*params);
    if (st != TSX_OK) return st;
    const tsx_enum_params &p = *params;
    const DevCode &g = code->d;

    // raw-set offsets per representative (host arithmetic on ball sizes)
    const int n_rep = g.n_rep;
    std::vector<long long> raw_off(n_rep + 1, 0);
    for (int r = 0; r < n_rep; r++) {
        long long nb = code->ball_ptr[r + 1] - code->ball_ptr[r];
        long long k = 1;
        if (p.max_size >= 2) k += nb;
        if (p.max_size >= 3) k += nb * (nb - 1) / 2;
        if (p.max_size >= 4) k += nb * (nb - 1) * (nb - 2) / 6;
        raw_off[r + 1] = raw_off[r] + k;
    }
    const long long raw_total = raw_off[n_rep];
    const int l = p.cycle_len / 2;
    const bool cycles = l > p.max_size;
    long long paths = 0, cyc_bound = 0;
    if (cycles) {
        paths = 1;
        for (int i = 0; i < l; i++) paths *= g.dv_max;
        for (int i = 0; i + 1 < l; i++) paths *= g.dc_max;
        if (paths > (1LL << 30)) return TSX_EUNSUPPORTED;
        cyc_bound = (long long)n_rep * 2048;
    }
    const long long cand_bound = raw_total + cyc_bound;
    if (cand_bound > (1LL << 31)) return TSX_ENOMEM;
    long long n_rec = cand_bound - p.cand_begin;
    if (p.cand_end >= 0) n_rec = std::min<long long>(n_rec, p.cand_end - p.cand_begin);
    if (n_rec < 0) n_rec = 0;

    if (!decode_fits(g, p.decoder)) return TSX_EUNSUPPORTED;
    if (p.list_mode && !list_fits(g, p.K)) return TSX_EUNSUPPORTED;

    tsx_ts_list *L = new tsx_ts_list();
    L->dry = dry;
    L->code = code;
    L->st = s;
    L->p = p;
    L->grid_sms = grid_sms > 0 ? std::min(grid_sms, code->num_sms) : code->num_sms;
    L->range_end = p.cand_end >= 0 ? std::min<long long>(p.cand_end, cand_bound) : cand_bound;
    if (dchunk > 0) {
        L->dchunk = dchunk;
        L->n_dchunks = std::max<long long>(1, (L->range_end - p.cand_begin + dchunk - 1) / dchunk);
    }
    L->n_rec = n_rec;
    L->events = events;
    L->raw_off = raw_off;
    L->raw_total = raw_total;
    L->cycles = cycles;
    L->cyc_l = l;
    L->paths = paths;
    // list mode: up to two sets per iteration of every failing candidate
    if (p.list_mode) {
        const long long want = std::max<long long>(1, n_rec) * (long long)(p.K + 1);
        L->cap = next_pow2(std::min<long long>(std::max<long long>(1 << 16, want), 1LL << 28));
        L->pool_cap = std::min<long long>(L->cap * 24, 0xfffffff0LL);
    } else {
        L->cap = next_pow2(std::max<long long>(1024, 2 * std::max<long long>(n_rec, 1)));
        L->pool_cap = std::max<long long>(1 << 20, 24 * n_rec);
    }
    if (L->pool_cap > 0xfffffff0LL) L->pool_cap = 0xfffffff0LL;
    DecodeParams &dp = L->dp;
    dp.decoder = p.decoder; dp.K = p.K; dp.base_llr = p.base_llr; dp.sat = p.sat;
    dp.alpha_num = p.alpha_num; dp.alpha_shift = p.alpha_shift; dp.amp_steps = p.amp_steps;
    dp.spa_clip = p.spa_clip; dp.spa_amax = p.spa_amax;

    L->n_chunks = cand_chunks(raw_total);
    L->d_raw_off = lalloc<long long>(L, n_rep + 1, s);
    L->d_chunk_cnt = lalloc<int>(L, L->n_chunks, s);
    L->d_chunk_off = lalloc<long long>(L, L->n_chunks + 1, s);
    int4 *d_cands = lalloc<int4>(L, cand_bound, s);
    L->b.cand_K = p.budget_wref > 0 ? lalloc<uint16_t>(L, cand_bound, s) : nullptr;
    L->cand_bound = cand_bound;
    L->d_cyc_cnt = cycles ? lalloc<int>(L, n_rep, s) : nullptr;
    L->d_cyc_off = cycles ? lalloc<long long>(L, n_rep + 1, s) : nullptr;
    EnumBuffers &b = L->b;
    b.cands = d_cands;
    b.cand_begin = p.cand_begin;
    b.cand_end = p.cand_end;
    b.record = 1;
    const long long nr = n_rec;  // the sieve reads the records, so they are always kept
    b.nw = (g.n + 31) / 32;
    b.xstar = lalloc<uint32_t>(L, (size_t)n_rec * b.nw, s);
    b.c_thr = lalloc<int>(L, nr, s);
    b.c_thr_f = lalloc<float>(L, nr, s);
    b.c_slot = lalloc<int>(L, nr, s);
    b.c_flags = lalloc<int>(L, nr, s);
    b.c_decodes = lalloc<int>(L, nr, s);
    b.c_iters = lalloc<int>(L, nr, s);
    b.tags = lalloc<unsigned long long>(L, L->cap, s);
    b.t_thr = lalloc<int>(L, L->cap, s);
    b.t_count = lalloc<int>(L, L->cap, s);
    b.cap_mask = (unsigned long long)(L->cap - 1);
    b.pool = lalloc<int>(L, L->pool_cap + 1, s);
    b.pool_cap = (unsigned long long)L->pool_cap;
    L->ctr = lalloc<Counters>(L, 1, s);
    b.ctr = L->ctr;
    b.queue = L->ctr ? &L->ctr->next_cand : nullptr;
    b.rec_base = p.cand_begin;
    // distinct sets: at most one per failing candidate, or (list mode) as many as the table holds
    const long long ts_cap = p.list_mode ? L->cap : std::min<long long>(L->cap, std::max<long long>(n_rec, 1));
    L->ts_off = lalloc<int>(L, ts_cap, s);
    L->ts_count = lalloc<int>(L, ts_cap, s);
    L->ts_thr = lalloc<int>(L, ts_cap, s);
    L->slot_map = lalloc<int>(L, L->cap, s);
    if (L->n_dchunks) L->d_queues = lalloc<unsigned long long>(L, L->n_dchunks, s);
    if (dry) {
        *out = L;
        return TSX_OK;
    }
    if (L->oom) {
        cudaGetLastError();
        release(L);
        delete L;
        return TSX_ENOMEM;
    }
    auto bail = [&](int code_) { release(L); delete L; return code_; };
    if (events)
        for (cudaEvent_t &e : L->ev)
            if (cudaEventCreate(&e) != cudaSuccess) return bail(TSX_ECUDA);
    if (cudaMemcpyAsync(L->d_raw_off, L->raw_off.data(), sizeof(long long) * (n_rep + 1), cudaMemcpyHostToDevice,
                        s) != cudaSuccess)
        return bail(TSX_ECUDA);
    *out = L;
    return TSX_OK;
}

static int record(tsx_ts_list *L, int i, cudaStream_t s) {
    if (!L->events) return TSX_OK;
    return cudaEventRecord(L->ev[i], s) == cudaSuccess ? TSX_OK : TSX_ECUDA;
}

// counters and table reset, candidate generation
static int enqueue_front(tsx_ts_list *L, cudaStream_t s) {
    const DevCode &g = L->code->d;
    EnumBuffers &b = L->b;
    L->st = s;
    L->fetched = false;
    if (record(L, 0, s) != TSX_OK) return TSX_ECUDA;
    if (cudaMemsetAsync(L->ctr, 0, sizeof(Counters), s) != cudaSuccess ||
        cudaMemsetAsync(b.tags, 0, sizeof(unsigned long long) * L->cap, s) != cudaSuccess ||
        cudaMemsetAsync(b.t_count, 0, sizeof(int) * L->cap, s) != cudaSuccess ||
        cudaMemsetAsync(b.t_thr, 0x7f, sizeof(int) * L->cap, s) != cudaSuccess ||
        (L->d_queues &&
         cudaMemsetAsync(L->d_queues, 0, sizeof(unsigned long long) * L->n_dchunks, s) != cudaSuccess))
        return TSX_ECUDA;
    CandArgs ca{};
    ca.code = g;
    ca.max_size = L->p.max_size;
    ca.raw_off = L->d_raw_off;
    ca.raw_total = L->raw_total;
    ca.chunk_count = L->d_chunk_cnt;
    ca.chunk_off = L->d_chunk_off;
    ca.cands = (int4 *)b.cands;
    ca.ctr = L->ctr;
    if (launch_cand_ball(ca, L->n_chunks, false, s) != cudaSuccess ||
        launch_scan(L->d_chunk_cnt, L->n_chunks, L->d_chunk_off, nullptr, L->ctr, !L->cycles, s) != cudaSuccess ||
        launch_cand_ball(ca, L->n_chunks, true, s) != cudaSuccess)
        return TSX_ECUDA;
    if (L->cycles) {
        CycleArgs cy{};
        cy.code = g;
        cy.l = L->cyc_l;
        cy.paths = L->paths;
        cy.count = L->d_cyc_cnt;
        cy.off = L->d_cyc_off;
        cy.cands = (int4 *)b.cands;
        cy.ctr = L->ctr;
        if (launch_cand_cycle(cy, false, s) != cudaSuccess ||
            launch_scan(L->d_cyc_cnt, g.n_rep, L->d_cyc_off, L->d_chunk_off + L->n_chunks, L->ctr, true, s) !=
                cudaSuccess ||
            launch_cand_cycle(cy, true, s) != cudaSuccess)
            return TSX_ECUDA;
    }
    if (L->b.cand_K && launch_budget(b.cands, L->cand_bound, L->code->vweight, L->p.K, L->p.budget_kmin,
                                     L->p.budget_wref, (uint16_t *)L->b.cand_K, L->ctr, s) != cudaSuccess)
        return TSX_ECUDA;
    return record(L, 1, s);
}

static int enqueue_decode(tsx_ts_list *L, cudaStream_t s) {
    const tsx_enum_params &p = L->p;
    if (!L->n_dchunks) {
        if (launch_decode(L->code->d, L->dp, L->b, p.warps_per_cta, 0, p.ctas_per_sm, L->grid_sms,
                          p.kernel == 1 ? 1 : 0, s) != cudaSuccess)
            return TSX_ECUDA;
        return TSX_OK;
    }
    // one launch per chunk: between launches the SMs can go to other streams
    for (long long k = 0; k < L->n_dchunks; k++) {
        EnumBuffers bk = L->b;
        bk.cand_begin = p.cand_begin + k * L->dchunk;
        bk.cand_end = std::min<long long>(bk.cand_begin + L->dchunk, L->range_end);
        bk.queue = L->d_queues + k;
        if (launch_decode(L->code->d, L->dp, bk, p.warps_per_cta, 0, p.ctas_per_sm, L->grid_sms,
                          p.kernel == 1 ? 1 : 0, s) != cudaSuccess)
            return TSX_ECUDA;
    }
    return TSX_OK;
}

// sieve, classification, dedupe, compaction
static int enqueue_back(tsx_ts_list *L, cudaStream_t s) {
    if (record(L, 2, s) != TSX_OK) return TSX_ECUDA;
    if (L->p.list_mode) {
        if (launch_list(L->code->d, L->dp, L->b, L->p.kstart, L->grid_sms, s) != cudaSuccess) return TSX_ECUDA;
    } else if (launch_sieve(L->code->d, L->b, L->p.decoder, L->grid_sms, s) != cudaSuccess) {
        return TSX_ECUDA;
    }
    if (record(L, 3, s) != TSX_OK) return TSX_ECUDA;
    if (launch_compact(L->b, L->n_rec, L->ts_off, L->ts_count, L->ts_thr, L->slot_map, s) != cudaSuccess)
        return TSX_ECUDA;
    return record(L, 4, s);
}

extern "C" int enumerate_ts(tsx_code *code, const tsx_enum_params *params, void *stream, tsx_ts_list **out) {
    if (!code || !params || !out) return TSX_EINVAL;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    tsx_ts_list *L = nullptr;
    int st = prepare_list(code, params, s, true, &L);
    if (st != TSX_OK) return st;
    if ((st = enqueue_front(L, s)) != TSX_OK || (st = enqueue_decode(L, s)) != TSX_OK ||
        (st = enqueue_back(L, s)) != TSX_OK) {
        release(L);
        delete L;
        return st;
    }
    *out = L;
    return TSX_OK;
}

// ---------------------------------------------------------------------------
// tile autotuner: times the decode on a prefix of the candidate list for each
// admissible (warps per codeword group, message storage) and keeps the fastest
// ---------------------------------------------------------------------------
extern "C" int tune_tile(tsx_code *code, const tsx_enum_params *params, void *stream, tsx_enum_params *tuned,
                         float *ms_best) {
    if (!code || !params || !tuned) return TSX_EINVAL;
    int st = check_params(*params);
    if (st != TSX_OK) return st;
    *tuned = *params;
    if (ms_best) *ms_best = -1.0f;
    if (params->decoder == TSX_DEC_SPA_F32 || params->kernel == 1) return TSX_OK;  // nothing to choose
    const DevCode &g = code->d;
    std::vector<int> decs{params->decoder};
    // int8 storage is exact when every check-to-variable message fits in 8 bits
    if (params->decoder == TSX_DEC_NMS_I16 && params->sat <= 169) decs.push_back(TSX_DEC_NMS_I8);
    int work = std::min(g.m, g.n);
    if (g.kind == TSX_CODE_QC) work = std::min(work, g.Z);
    // 0: the automatic shape (as many codeword groups as fit, the warps shared among them)
    std::vector<int> Gs{0, 1};
    for (int G = 2; G <= 8 && G * 32 <= std::max(32, work); G *= 2) Gs.push_back(G);
    tsx_enum_params t = *params;
    t.record_candidates = 0;
    t.cand_begin = 0;
    t.cand_end = (long long)code->num_sms * 256;
    t.ctas_per_sm = 0;
    float best = -1.0f;
    bool warm = false;
    for (int dec : decs)
        for (int G : Gs) {
            t.decoder = dec;
            t.warps_per_cta = G;
            t.kernel = 0;
            for (int rep = warm ? 1 : 0; rep < 2; rep++) {
                tsx_ts_list *L = nullptr;
                st = enumerate_ts(code, &t, stream, &L);
                if (st == TSX_EUNSUPPORTED) break;
                if (st != TSX_OK) return st;
                tsx_enum_stats es;
                st = ts_list_stats(L, &es);
                free_ts_list(L);
                if (st != TSX_OK) return st;
                warm = true;
                if (rep == 1 && (best < 0.0f || es.ms_decode < best)) {
                    best = es.ms_decode;
                    tuned->decoder = dec;
                    tuned->warps_per_cta = G;
                }
            }
        }
    if (ms_best) *ms_best = best;
    return TSX_OK;
}

// ---------------------------------------------------------------------------
// batches: several codes, one multi-code decode launch
// ---------------------------------------------------------------------------
struct tsx_batch {
    std::vector<tsx_ts_list *> lists;
    BatchArgs *items = nullptr;  // host copy, passed by value at each launch
    int n_items = 0;             // codes in the multi-code launch
    std::vector<bool> own;       // codes decoded by a launch of their own
    LaunchShape sh{};
    int variant = 0;
    bool multi = false;
};

extern "C" void batch_free(tsx_batch *B) {
    if (!B) return;
    for (tsx_ts_list *L : B->lists) free_ts_list(L);
    delete B->items;
    delete B;
}

extern "C" int batch_create(tsx_code *const *codes, const tsx_enum_params *params, int32_t n, void *stream,
                            tsx_batch **out) {
    if (!codes || !params || !out || n <= 0) return TSX_EINVAL;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    tsx_batch *B = new tsx_batch();
    for (int i = 0; i < n; i++) {
        if (!codes[i]) { batch_free(B); return TSX_EINVAL; }
        tsx_ts_list *L = nullptr;
        const int st = prepare_list(codes[i], &params[i], s, false, &L);
        if (st != TSX_OK) { batch_free(B); return st; }
        B->lists.push_back(L);
    }
    std::vector<const DevCode *> gs(n);
    std::vector<DecodeParams> dps(n);
    std::vector<EnumBuffers> bs(n);
    std::vector<BatchItem> items(n);
    std::vector<int> greq(n);
    bool all_auto = true;
    for (int i = 0; i < n; i++) {
        greq[i] = params[i].warps_per_cta;
        gs[i] = &B->lists[i]->code->d;
        dps[i] = B->lists[i]->dp;
        bs[i] = B->lists[i]->b;
        all_auto = all_auto && params[i].kernel != 1;
    }
    if (all_auto && n <= kMaxBatch &&
        plan_batch(gs.data(), dps.data(), bs.data(), greq.data(), n, codes[0]->num_sms, items.data(), &B->sh,
                   &B->variant)) {
        B->items = new BatchArgs();
        for (int i = 0; i < n; i++) {
            B->own.push_back(items[i].scalar != 0);
            if (!items[i].scalar) B->items->it[B->n_items++] = items[i];
        }
        B->multi = B->n_items > 0;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { batch_free(B); return TSX_ECUDA; }
    *out = B;
    return TSX_OK;
}

extern "C" int batch_run(tsx_batch *B, void *stream) {
    if (!B) return TSX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int st;
    for (tsx_ts_list *L : B->lists)
        if ((st = enqueue_front(L, s)) != TSX_OK) return st;
    if (B->multi) {
        if (launch_batch(*B->items, B->n_items, B->variant, B->sh, s) != cudaSuccess) return TSX_ECUDA;
        for (size_t i = 0; i < B->lists.size(); i++)
            if (B->own[i] && (st = enqueue_decode(B->lists[i], s)) != TSX_OK) return st;
    } else {
        for (tsx_ts_list *L : B->lists)
            if ((st = enqueue_decode(L, s)) != TSX_OK) return st;
    }
    for (tsx_ts_list *L : B->lists)
        if ((st = enqueue_back(L, s)) != TSX_OK) return st;
    return TSX_OK;
}

extern "C" int batch_size(const tsx_batch *B) { return B ? (int)B->lists.size() : 0; }

extern "C" int batch_multi_launch(const tsx_batch *B) { return B && B->multi ? 1 : 0; }

extern "C" int batch_decode_launches(const tsx_batch *B) {
    if (!B) return 0;
    if (!B->multi) return (int)B->lists.size();
    int n = 1;
    for (bool own : B->own) n += own ? 1 : 0;
    return n;
}

extern "C" int batch_view(tsx_batch *B, int32_t i, tsx_ts_view *view) {
    if (!B || i < 0 || i >= (int)B->lists.size()) return TSX_EINVAL;
    return ts_list_view(B->lists[i], view);
}

extern "C" int batch_stats(tsx_batch *B, tsx_enum_stats *total) {
    if (!B || !total) return TSX_EINVAL;
    memset(total, 0, sizeof(*total));
    int ret = TSX_OK;
    for (tsx_ts_list *L : B->lists) {
        tsx_enum_stats s;
        const int st = ts_list_stats(L, &s);
        if (st != TSX_OK && ret == TSX_OK) ret = st;
        total->n_cand += s.n_cand;
        total->n_cand_total += s.n_cand_total;
        total->n_ts += s.n_ts;
        total->decodes += s.decodes;
        total->iterations += s.iterations;
        total->edge_updates += s.edge_updates;
        total->acyclic += s.acyclic;
        total->converged += s.converged;
        total->converged_iterations += s.converged_iterations;
        total->list_patterns += s.list_patterns;
        total->list_iterations += s.list_iterations;
    }
    return ret;
}

static int fetch_counters(tsx_ts_list *L, Counters &c) {
    if (cudaStreamSynchronize(L->st) != cudaSuccess) return TSX_ECUDA;
    if (cudaMemcpy(&c, L->ctr, sizeof(Counters), cudaMemcpyDeviceToHost) != cudaSuccess) return TSX_ECUDA;
    return TSX_OK;
}

static void fill_stats(tsx_ts_list *L, const Counters &c, tsx_enum_stats &s) {
    long long total = (long long)c.n_cand_total;
    long long end = L->p.cand_end < 0 || L->p.cand_end > total ? total : L->p.cand_end;
    s.n_cand = std::max<long long>(0, end - L->p.cand_begin);
    s.n_cand_total = total;
    s.n_ts = c.n_ts;
    s.decodes = (int64_t)c.decodes;
    s.iterations = (int64_t)c.iterations;
    s.edge_updates = (int64_t)c.edge_updates;
    s.acyclic = (int64_t)c.acyclic;
    s.converged = (int64_t)c.ok_decodes;
    s.converged_iterations = (int64_t)c.ok_iters;
    s.list_kstart = (int64_t)c.list_kstart;
    s.list_patterns = (int64_t)c.list_patterns;
    s.list_iterations = (int64_t)c.list_iters;
    float ms = 0.0f;
    if (L->ev[4] && cudaEventElapsedTime(&ms, L->ev[0], L->ev[4]) == cudaSuccess) s.ms_total = ms;
    if (L->ev[1] && cudaEventElapsedTime(&ms, L->ev[0], L->ev[1]) == cudaSuccess) s.ms_candidates = ms;
    if (L->ev[2] && cudaEventElapsedTime(&ms, L->ev[1], L->ev[2]) == cudaSuccess) s.ms_decode = ms;
    if (L->ev[3] && cudaEventElapsedTime(&ms, L->ev[2], L->ev[3]) == cudaSuccess) s.ms_sieve = ms;
}

extern "C" int ts_list_stats(tsx_ts_list *L, tsx_enum_stats *stats) {
    if (!L || !stats) return TSX_EINVAL;
    if (L->fetched) { *stats = L->stats; return L->fetch_status; }
    Counters c;
    int st = fetch_counters(L, c);
    if (st != TSX_OK) return st;
    fill_stats(L, c, *stats);
    if (c.err & (kErrPoolOverflow | kErrTableFull | kErrCandOverflow | kErrCycleOverflow)) return TSX_ENOMEM;
    return TSX_OK;
}

static int do_fetch(tsx_ts_list *L) {
    Counters c;
    int st = fetch_counters(L, c);
    if (st != TSX_OK) return st;
    fill_stats(L, c, L->stats);
    const long long nts = c.n_ts;
    std::vector<int> off(nts), cnt(nts), thr(nts);
    const unsigned long long pool_used = c.pool_top + 1 < (unsigned long long)L->pool_cap + 1
                                             ? c.pool_top + 1
                                             : (unsigned long long)L->pool_cap + 1;
    std::vector<int> pool(pool_used);
    if (nts) {
        CK(cudaMemcpy(off.data(), L->ts_off, sizeof(int) * nts, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(cnt.data(), L->ts_count, sizeof(int) * nts, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(thr.data(), L->ts_thr, sizeof(int) * nts, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(pool.data(), L->b.pool, sizeof(int) * pool_used, cudaMemcpyDeviceToHost));
    }
    // sort by (a, b, key)
    std::vector<int> perm(nts);
    std::iota(perm.begin(), perm.end(), 0);
    auto less = [&](int x, int y) {
        const int *px = &pool[off[x]], *py = &pool[off[y]];
        if (px[0] != py[0]) return px[0] < py[0];
        if (px[1] != py[1]) return px[1] < py[1];
        return std::lexicographical_compare(px + kPoolHdr, px + kPoolHdr + px[0], py + kPoolHdr, py + kPoolHdr + py[0]);
    };
    std::sort(perm.begin(), perm.end(), less);
    std::vector<int> rank(nts);
    for (long long i = 0; i < nts; i++) rank[perm[i]] = (int)i;
    const bool spa = L->p.decoder == TSX_DEC_SPA_F32;
    L->a.resize(nts); L->b_.resize(nts); L->orbit.resize(nts); L->count.resize(nts);
    L->thr.resize(nts); L->thr_f.resize(nts); L->flags.resize(nts); L->var_off.resize(nts + 1);
    L->vars.clear();
    long long vo = 0;
    for (long long i = 0; i < nts; i++) {
        const int x = perm[i];
        const int *px = &pool[off[x]];
        L->a[i] = px[0]; L->b_[i] = px[1]; L->orbit[i] = px[2]; L->flags[i] = px[3];
        L->count[i] = cnt[x];
        if (spa) {
            float f;
            memcpy(&f, &thr[x], 4);
            L->thr_f[i] = f;
            L->thr[i] = -1;
        } else {
            L->thr[i] = thr[x];
            L->thr_f[i] = -1.0f;
        }
        L->var_off[i] = vo;
        L->vars.insert(L->vars.end(), px + kPoolHdr, px + kPoolHdr + px[0]);
        vo += px[0];
    }
    L->var_off[nts] = vo;
    const long long ncand = L->p.record_candidates ? std::min<long long>(L->stats.n_cand, L->n_rec) : 0;
    L->cvars.resize(4 * ncand); L->cthr.resize(ncand); L->cthr_f.resize(ncand); L->cts.resize(ncand);
    L->cflags.resize(ncand); L->cdec.resize(ncand); L->cit.resize(ncand);
    if (ncand) {
        CK(cudaMemcpy(L->cvars.data(), L->b.cands + L->p.cand_begin, sizeof(int4) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cthr.data(), L->b.c_thr, sizeof(int) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cthr_f.data(), L->b.c_thr_f, sizeof(float) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cts.data(), L->b.c_slot, sizeof(int) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cflags.data(), L->b.c_flags, sizeof(int) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cdec.data(), L->b.c_decodes, sizeof(int) * ncand, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(L->cit.data(), L->b.c_iters, sizeof(int) * ncand, cudaMemcpyDeviceToHost));
        for (long long i = 0; i < ncand; i++)
            if (L->cts[i] >= 0) L->cts[i] = rank[L->cts[i]];
    }
    if (c.err & (kErrPoolOverflow | kErrTableFull | kErrCandOverflow | kErrCycleOverflow)) return TSX_ENOMEM;
    return TSX_OK;
}

extern "C" int ts_list_view(tsx_ts_list *L, tsx_ts_view *v) {
    if (!L || !v) return TSX_EINVAL;
    if (!L->fetched) {
        L->fetch_status = do_fetch(L);
        L->fetched = true;
    }
    memset(v, 0, sizeof(*v));
    v->stats = L->stats;
    v->n_ts = (int64_t)L->a.size();
    v->a = L->a.data(); v->b = L->b_.data(); v->orbit = L->orbit.data(); v->count = L->count.data();
    v->thr = L->thr.data(); v->flags = L->flags.data(); v->thr_f = L->thr_f.data();
    v->var_off = L->var_off.data(); v->vars = L->vars.data();
    v->n_cand = (int64_t)L->cthr.size();
    v->cand_vars = L->cvars.data(); v->cand_thr = L->cthr.data(); v->cand_ts = L->cts.data();
    v->cand_flags = L->cflags.data(); v->cand_decodes = L->cdec.data(); v->cand_iters = L->cit.data();
    v->cand_thr_f = L->cthr_f.data();
    return L->fetch_status;
}

extern "C" void free_ts_list(tsx_ts_list *L) {
    if (!L) return;
    release(L);
    cudaStreamSynchronize(L->st);
    delete L;
}

// ---------------------------------------------------------------------------
// hooks of the serving runtime (server.cu)
// ---------------------------------------------------------------------------
namespace tsx {

int list_bytes(tsx_code *code, const tsx_enum_params *params, long long dchunk, long long *bytes,
               long long *cand_bound) {
    tsx_ts_list *L = nullptr;
    const int st = prepare_list(code, params, nullptr, false, &L, dchunk, 0, true);
    if (st != TSX_OK) return st;
    *bytes = L->bytes;
    if (cand_bound) *cand_bound = std::max<long long>(0, L->range_end - L->p.cand_begin);
    delete L;
    return TSX_OK;
}

long long list_cand_bound(const tsx_ts_list *L) { return L->range_end - L->p.cand_begin; }

int list_start(tsx_code *code, const tsx_enum_params *params, cudaStream_t s, long long dchunk, int grid_sms,
               tsx_ts_list **out) {
    tsx_ts_list *L = nullptr;
    int st = prepare_list(code, params, s, true, &L, dchunk, grid_sms, false);
    if (st != TSX_OK) return st;
    if ((st = enqueue_front(L, s)) != TSX_OK || (st = enqueue_decode(L, s)) != TSX_OK ||
        (st = enqueue_back(L, s)) != TSX_OK) {
        release(L);
        delete L;
        return st;
    }
    *out = L;
    return TSX_OK;
}

// After the list's stream has passed its last kernel: copy the results to
// the host and give the device memory back (stream-ordered).  The list stays
// valid for ts_list_view(); delete it with list_delete().
int list_finish(tsx_ts_list *L) {
    if (!L->fetched) {
        L->fetch_status = do_fetch(L);
        L->fetched = true;
    }
    release(L);
    return L->fetch_status;
}

void list_delete(tsx_ts_list *L) {
    if (!L) return;
    release(L);
    delete L;
}

}  // namespace tsx
