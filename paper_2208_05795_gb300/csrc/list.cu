// list.cu -- the ordered list of trapping sets of Sec. III, as the second
// stage of a two-stage schedule.
//
// The first stage is the ordinary enumeration decode: every candidate's
// bisection, which leaves the threshold amplitude of each failing candidate
// (and counts the decodes that converged and their iterations).  The second
// stage takes only the failing candidates: one group of warps replays the
// decode at the candidate's threshold (the same decoder, so the same x_k),
// and for every iteration k from kstart to K_last forms X_k = supp(x_k) u I,
// S1(x_k) = Tree(X_k) and S2(x_k) = Tree(TS(X_k)); every non-empty one is a
// trapping set and goes into the hash table with its canonical key, each set
// counted once per candidate.  An x_k equal to the previous one is not
// sieved again (it gives the same two sets).  kstart is floor(girth/2), a
// given iteration, or -- the paper's scheduler -- ceil of the average
// iteration count of the first stage's converged decodes, read on the device
// from the first stage's counters.
#include "decode_impl.cuh"

namespace tsx {
namespace {

struct ListLayout {
    int tables_bytes;
    int r_off, p_off, s_off, xk_off, xp_off, deg_off, l_off, key_off, seen_off, misc_off;
    int slot_bytes;
};

ListLayout list_layout(const DevCode &g, int K) {
    ListLayout L{};
    L.tables_bytes = al16(tab_offsets(g, false).total);
    const int nw = (g.n + 31) / 32;
    const int nmsg = g.kind == TSX_CODE_QC ? g.E : g.m * g.dc_max;
    int x = 0;
    L.r_off = x; x += al16(nmsg * 2);
    L.p_off = x; x += al16(g.n * 2);
    L.s_off = x; x += al16(nw * 4);
    L.xk_off = x; x += al16(nw * 4);
    L.xp_off = x; x += al16(nw * 4);
    L.deg_off = x; x += al16(g.m * 4);
    L.l_off = x; x += al16(g.n * 2);
    L.key_off = x; x += al16(g.n * 2);
    L.seen_off = x; x += al16(2 * (K + 1) * 4);  // at most two sets per iteration
    L.misc_off = x; x += al16((int)sizeof(Misc));
    L.slot_bytes = x;
    return L;
}

constexpr int kSmemCta = 226 * 1024;
// up to 20 warps a CTA: the second stage is latency and barrier bound, and
// one group more than 16 warps allow fits the shared memory of the QC codes
constexpr int kListWarps = 20;

template <int DCMAX, bool QC>
__global__ void __launch_bounds__(32 * kListWarps) list_kernel(DevCode g, DecodeParams dp, EnumBuffers b, ListLayout lay, int G,
                                                    int kstart_req) {
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
    int16_t *P = (int16_t *)(slot + lay.p_off);
    int16_t *R = (int16_t *)(slot + lay.r_off);
    uint32_t *S = (uint32_t *)(slot + lay.s_off);
    uint32_t *Xk = (uint32_t *)(slot + lay.xk_off);
    uint32_t *Xp = (uint32_t *)(slot + lay.xp_off);
    int *deg = (int *)(slot + lay.deg_off);
    uint16_t *L = (uint16_t *)(slot + lay.l_off);
    uint16_t *key = (uint16_t *)(slot + lay.key_off);
    int *seen = (int *)(slot + lay.seen_off);
    Decoder<DecNms16, DCMAX, QC> dec{g, sg, gp, dp, P, R};
    Sieve<QC> sv{g, sg, gp};

    // the first iteration of the lists
    int kstart = kstart_req;
    if (kstart == 0) {
        kstart = g.wstart;
    } else if (kstart < 0) {
        const unsigned long long ok = b.ctr->ok_decodes, okit = b.ctr->ok_iters;
        kstart = ok ? (int)((okit + ok - 1) / ok) : g.wstart;
        if (kstart < 1) kstart = 1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) b.ctr->list_kstart = (unsigned long long)kstart;

    const int nw = (g.n + 31) >> 5;
    const long long total = (long long)b.ctr->n_cand_total;
    const long long end = b.cand_end < 0 || b.cand_end > total ? total : b.cand_end;
    const long long n = end - b.cand_begin;
    const int Lbase = clampi(dp.base_llr, -dp.sat, dp.sat);
    long long my_pat = 0, my_it = 0;

    while (true) {
        if (gp.gt == 0) misc->bcast[0] = (long long)atomicAdd(&b.ctr->next_sieve, 1ull);
        gp.sync();
        const long long o = misc->bcast[0];
        gp.sync();
        if (o >= n) break;
        const int thr = b.c_thr[o];
        if (thr < 0) continue;  // no failure: not in the second stage
        const int4 I4 = b.cands[b.cand_begin + o];
        const int I[4] = {I4.x, I4.y, I4.z, I4.w};
        const int nI = (I4.x >= 0) + (I4.y >= 0) + (I4.z >= 0) + (I4.w >= 0);
        const int Limp = clampi(dp.base_llr - thr, -dp.sat, dp.sat);
        const int Kc = cand_limit(dp, b, b.cand_begin + o);
        if (gp.gt == 0) misc->ints[0] = 0;  // sets this candidate has counted
        for (int v = gp.gt; v < g.n; v += gp.T) P[v] = (int16_t)Lbase;
        gp.sync();
        if (gp.gt < nI) P[I[gp.gt]] = (int16_t)Limp;
        gp.sync();
        bool have_prev = false;
        bool first = true;
        int k = 0;
        while (true) {
            const int u = dec.check_pass(first, k < Kc);  // u_k of x_k = [P_k < 0]; R <- R_{k+1}
            first = false;
            if (k >= kstart) {
                dec.save_x(Xk);
                gp.sync();
                int diff = 0;
                if (have_prev)
                    for (int w = gp.gt; w < nw; w += gp.T) diff |= Xk[w] != Xp[w];
                diff = gp.sum(diff);
                if (!have_prev || diff) {
                    my_pat++;
                    for (int part = 1; part <= 2; part++) {
                        // S1: Tree(X_k); S2: Tree(TS(X_k))
                        sv.load_x(S, Xk, I, nI, deg);
                        if (part == 2) {
                            sv.closure(S, deg);
                            gp.sync();
                            sv.count_deg(S, deg);
                            gp.sync();
                        }
                        sv.peel(S, deg);
                        const int a = sv.popcount(S);
                        if (a == 0) continue;
                        int bb, elem;
                        sv.classify(deg, bb, elem);
                        if (gp.gw == 0) {
                            list_bits(S, g.n, L, lane);
                            const int orbit = canon_key(g, L, a, S, key, misc->seg, lane);
                            const long long ts = ts_insert(b, key, a, bb, orbit, elem | (part << 1), lane);
                            if (lane == 0 && ts >= 0) {
                                const int cnt = misc->ints[0];
                                bool dup = false;
                                for (int i = 0; i < cnt && !dup; i++) dup = seen[i] == (int)ts;
                                if (!dup) {
                                    seen[cnt] = (int)ts;
                                    misc->ints[0] = cnt + 1;
                                    atomicMin(&b.t_thr[ts], thr);
                                    atomicAdd(&b.t_count[ts], 1);
                                }
                            }
                        }
                        gp.sync();
                    }
                    uint32_t *t = Xk;
                    Xk = Xp;
                    Xp = t;
                    have_prev = true;
                }
            }
            if (u == 0 || k == Kc) break;
            dec.vn_pass(Lbase);
            gp.sync();
            if (gp.gt < nI) P[I[gp.gt]] = (int16_t)dec.posterior(I[gp.gt], Limp);
            gp.sync();
            k++;
        }
        my_it += k;
    }
    if (gp.gt == 0) {
        atomicAdd(&b.ctr->list_patterns, (unsigned long long)my_pat);
        atomicAdd(&b.ctr->list_iters, (unsigned long long)my_it);
    }
}

struct ListShape {
    ListLayout lay;
    int G, groups, smem;
};

bool list_shape(const DevCode &g, int K, ListShape *sh) {
    sh->lay = list_layout(g, K);
    const int fit = (kSmemCta - sh->lay.tables_bytes) / sh->lay.slot_bytes;
    if (fit < 1) return false;
    int work = g.m < g.n ? g.m : g.n;
    int G = work / 256;
    if (G < 1) G = 1;
    if (G > 4) G = 4;
    int groups = kListWarps / G;
    if (groups > fit) groups = fit;
    if (G > 1 && groups > 15) groups = 15;
    sh->G = G;
    sh->groups = groups;
    sh->smem = sh->lay.tables_bytes + groups * sh->lay.slot_bytes;
    return true;
}

template <class Kern>
cudaError_t launch_list_t(Kern k, const ListShape &sh, int num_sms, cudaStream_t st, const DevCode &g,
                          const DecodeParams &dp, const EnumBuffers &b, int kstart) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem);
    if (e != cudaSuccess) return e;
    const int threads = sh.groups * sh.G * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, sh.smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    k<<<occ * num_sms, threads, sh.smem, st>>>(g, dp, b, sh.lay, sh.G, kstart);
    return cudaGetLastError();
}

}  // namespace

bool list_fits(const DevCode &g, int K) {
    ListShape sh;
    return list_shape(g, K, &sh);
}

cudaError_t launch_list(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, int kstart, int num_sms,
                        cudaStream_t st) {
    ListShape sh;
    if (!list_shape(g, dp.K, &sh)) return cudaErrorInvalidConfiguration;
    const bool qc = g.kind == TSX_CODE_QC;
    if (g.dc_max <= 8)
        return qc ? launch_list_t(list_kernel<8, true>, sh, num_sms, st, g, dp, b, kstart)
                  : launch_list_t(list_kernel<8, false>, sh, num_sms, st, g, dp, b, kstart);
    return qc ? launch_list_t(list_kernel<32, true>, sh, num_sms, st, g, dp, b, kstart)
              : launch_list_t(list_kernel<32, false>, sh, num_sms, st, g, dp, b, kstart);
}

}  // namespace tsx
