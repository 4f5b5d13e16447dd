// decode_impl.cuh -- the persistent impulse-decoding kernel (instantiated
// per decoder in decode_i16.cu, decode_i8.cu and decode_spa.cu).
//
// One group of G warps owns one codeword slot in shared memory and runs,
// for each candidate impulse set it pops from a device work queue:
//   * the amplitude bisection (Cole's error impulse, Sec. III): a decode at
//     the largest amplitude, then up to s halvings keeping the failing end;
//   * each decode: flooding message passing from the all-zero codeword with
//     L_v = base everywhere except the impulse nodes, syndrome early exit,
//     and tracking of the error pattern x_k with the fewest unsatisfied
//     checks u_k = w_H(H x_k) from iteration floor(girth/2) on (Sec. III);
//   * on failure: the sieve S1 = Tree(X), else S2 = Tree(TS(X)), with
//     X = supp(x*) u I (Sec. III), the (a,b) classification (Sec. II), the
//     canonical form under the circulant shift and orbit size, and an
//     insert into the device hash table of distinct trapping sets.
// Messages never leave shared memory: per codeword the check-to-variable
// messages R[E] and posteriors P[n]; the variable-to-check messages are
// recomputed as clamp(P_v - r) when a check reads them.  Neighbour indices
// of QC codes come from the exponent matrix: (r + a) mod Z.
#pragma once
#include "graph.cuh"
#include "kernels.cuh"

namespace tsx {
namespace {  // each decoder translation unit gets its own copy

// ---------------------------------------------------------------------------
// decoder policies
// ---------------------------------------------------------------------------
struct DecNms16 {
    using msg = int16_t;
    using post = int16_t;
    using lv = int;
    static constexpr bool kFloat = false;
};
struct DecNms8 {
    using msg = int8_t;
    using post = int16_t;
    using lv = int;
    static constexpr bool kFloat = false;
};
struct DecSpa {
    using msg = float;
    using post = float;
    using lv = float;
    static constexpr bool kFloat = true;
};

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

struct TabOff {
    int rdeg, reoff, rjz, rs, cdeg, ceoff, cs, ciz;
    int c_ptr, c_vn, v_ptr, v_edge;
    int total;
};

// pair = the tables of the two-codeword kernels, which have no variable-node
// pass and so no per-variable edge lists (general codes)
__host__ __device__ inline TabOff tab_offsets(const DevCode &g, bool pair = false) {
    TabOff o{};
    int x = 0;
    if (g.kind == TSX_CODE_QC) {
        o.rdeg = x; x += al16(g.m_b * 2);
        o.reoff = x; x += al16(g.m_b * 4);
        o.rjz = x; x += al16(g.m_b * g.dc_max * 4);
        o.rs = x; x += al16(g.m_b * g.dc_max * 2);
        o.cdeg = x; x += al16(g.n_b * 2);
        o.ceoff = x; x += al16(g.n_b * g.dv_max * 4);
        o.cs = x; x += al16(g.n_b * g.dv_max * 2);
        o.ciz = x; x += al16(g.n_b * g.dv_max * 4);
    } else {
        o.c_ptr = x; x += al16((g.m + 1) * 2);
        o.c_vn = x; x += al16(g.E * 2);
        o.v_ptr = x; x += al16((g.n + 1) * 2);
        if (!pair) { o.v_edge = x; x += al16(g.E * 2); }
    }
    o.total = x;
    return o;
}

struct SGraph {
    const int16_t *rdeg;
    const int32_t *reoff, *rjz;
    const int16_t *rs, *cdeg;
    const int32_t *ceoff;
    const int16_t *cs;
    const int32_t *ciz;
    const uint16_t *c_ptr, *c_vn, *v_ptr, *v_edge;
};

__device__ void copy_bytes(void *dst, const void *src, int bytes) {
    // 16-byte vector copies when both ends allow, else bytes
    const int n16 = bytes >> 4;
    const int4 *s4 = (const int4 *)src;
    int4 *d4 = (int4 *)dst;
    if ((((uintptr_t)src) & 15) == 0) {
        for (int i = threadIdx.x; i < n16; i += blockDim.x) d4[i] = __ldg(s4 + i);
        for (int i = (n16 << 4) + threadIdx.x; i < bytes; i += blockDim.x)
            ((unsigned char *)dst)[i] = ((const unsigned char *)src)[i];
    } else {
        for (int i = threadIdx.x; i < bytes; i += blockDim.x)
            ((unsigned char *)dst)[i] = ((const unsigned char *)src)[i];
    }
}

__device__ SGraph load_tables(const DevCode &g, unsigned char *sm, bool pair = false) {
    TabOff o = tab_offsets(g, pair);
    SGraph s{};
    if (g.kind == TSX_CODE_QC) {
        copy_bytes(sm + o.rdeg, g.rdeg, g.m_b * 2);
        copy_bytes(sm + o.reoff, g.reoff, g.m_b * 4);
        copy_bytes(sm + o.rjz, g.rjz, g.m_b * g.dc_max * 4);
        copy_bytes(sm + o.rs, g.rs, g.m_b * g.dc_max * 2);
        copy_bytes(sm + o.cdeg, g.cdeg, g.n_b * 2);
        copy_bytes(sm + o.ceoff, g.ceoff, g.n_b * g.dv_max * 4);
        copy_bytes(sm + o.cs, g.cs, g.n_b * g.dv_max * 2);
        copy_bytes(sm + o.ciz, g.ciz, g.n_b * g.dv_max * 4);
        s.rdeg = (const int16_t *)(sm + o.rdeg);
        s.reoff = (const int32_t *)(sm + o.reoff);
        s.rjz = (const int32_t *)(sm + o.rjz);
        s.rs = (const int16_t *)(sm + o.rs);
        s.cdeg = (const int16_t *)(sm + o.cdeg);
        s.ceoff = (const int32_t *)(sm + o.ceoff);
        s.cs = (const int16_t *)(sm + o.cs);
        s.ciz = (const int32_t *)(sm + o.ciz);
    } else {
        copy_bytes(sm + o.c_ptr, g.c_ptr, (g.m + 1) * 2);
        copy_bytes(sm + o.c_vn, g.c_vn, g.E * 2);
        copy_bytes(sm + o.v_ptr, g.v_ptr, (g.n + 1) * 2);
        s.c_ptr = (const uint16_t *)(sm + o.c_ptr);
        s.c_vn = (const uint16_t *)(sm + o.c_vn);
        s.v_ptr = (const uint16_t *)(sm + o.v_ptr);
        if (!pair) {
            copy_bytes(sm + o.v_edge, g.v_edge, g.E * 2);
            s.v_edge = (const uint16_t *)(sm + o.v_edge);
        }
    }
    return s;
}

// ---------------------------------------------------------------------------
// a group of G warps working on one codeword
// ---------------------------------------------------------------------------
struct Grp {
    int G, T, gt, lane, gw, bar;
    int *red;  // reduction scratch (shared): [0, 16) for sum(), [16, 32) for sum_pass()
    __device__ __forceinline__ void sync() const {
        if (G == 1) __syncwarp();
        else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(T) : "memory");
    }
    __device__ __forceinline__ int sum(int x) const {
        x = __reduce_add_sync(0xffffffffu, x);
        if (G == 1) {
            __syncwarp();
            return x;
        }
        if (lane == 0) red[gw] = x;
        sync();
        int s = 0;
        for (int w = 0; w < G; w++) s += red[w];
        sync();
        return s;
    }
    // the same on the second scratch bank without the closing barrier: the
    // caller passes a group barrier before its next sum_pass
    __device__ __forceinline__ int sum_pass(int x) const {
        x = __reduce_add_sync(0xffffffffu, x);
        if (G == 1) {
            __syncwarp();
            return x;
        }
        if (lane == 0) red[16 + gw] = x;
        sync();
        int s = 0;
        for (int w = 0; w < G; w++) s += red[16 + w];
        return s;
    }
};

// ---------------------------------------------------------------------------
// single-precision tanh / atanh of the sum-product check update, from their
// series with IEEE-rounded adds, multiplies and divides only (no fused
// multiply-add), so the result is the same on every conforming machine:
//   expm1(x), x >= 0: k = rint(x/ln2), r = (x - k ln2_hi) - k ln2_lo
//     (Cody-Waite reduction), expm1(r) = sum_{i=1..9} r^i/i! by Horner,
//     expm1(x) = 2^k (expm1(r) + 1) - 1 if k != 0;
//   tanh(y) = sgn(y) e / (e + 2), e = expm1(2|y|);
//   atanh(p) = sgn(p) sum_{j=0..8} a^(2j+1)/(2j+1) for a = |p| < 1/4, else
//     sgn(p) log(t)/2, t = (1+a)/(1-a) = m 2^e with m in [sqrt(1/2),
//     sqrt(2)), log t = e ln2 + 2 sum_{j=0..6} s^(2j+1)/(2j+1),
//     s = (m-1)/(m+1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float hsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float hmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float hdiv(float a, float b) { return __fdiv_rn(a, b); }

__device__ __forceinline__ float spa_expm1_pos(float x) {
    const float k = rintf(hmul(x, 0x1.715476p+0f));
    const float r = hsub(hsub(x, hmul(k, 0x1.62e4p-1f)), hmul(k, 0x1.7f7d1cp-20f));
    float p = 0x1.71de3ap-19f;  // 1/9!
    p = hadd(hmul(p, r), 0x1.a01a02p-16f);
    p = hadd(hmul(p, r), 0x1.a01a02p-13f);
    p = hadd(hmul(p, r), 0x1.6c16c2p-10f);
    p = hadd(hmul(p, r), 0x1.111112p-7f);
    p = hadd(hmul(p, r), 0x1.555556p-5f);
    p = hadd(hmul(p, r), 0x1.555556p-3f);
    p = hadd(hmul(p, r), 0.5f);
    p = hadd(hmul(p, r), 1.0f);
    p = hmul(p, r);
    if (k == 0.0f) return p;
    return hsub(ldexpf(hadd(p, 1.0f), (int)k), 1.0f);
}

__device__ __forceinline__ float spa_tanhf(float y) {
    const float a = fabsf(y);
    const float e = spa_expm1_pos(hadd(a, a));
    const float t = hdiv(e, hadd(e, 2.0f));
    return y < 0.0f ? -t : t;
}

__device__ __forceinline__ float spa_atanhf(float p) {
    const float a = fabsf(p);
    float r;
    if (a < 0.25f) {
        const float a2 = hmul(a, a);
        float q = 0x1.e1e1e2p-5f;  // 1/17
        q = hadd(hmul(q, a2), 0x1.111112p-4f);
        q = hadd(hmul(q, a2), 0x1.3b13b2p-4f);
        q = hadd(hmul(q, a2), 0x1.745d18p-4f);
        q = hadd(hmul(q, a2), 0x1.c71c72p-4f);
        q = hadd(hmul(q, a2), 0x1.24924ap-3f);
        q = hadd(hmul(q, a2), 0x1.99999ap-3f);
        q = hadd(hmul(q, a2), 0x1.555556p-2f);
        q = hadd(hmul(q, a2), 1.0f);
        r = hmul(q, a);
    } else {
        const float t = hdiv(hadd(1.0f, a), hsub(1.0f, a));
        int e;
        float m = frexpf(t, &e);
        if (m < 0x1.6a09e6p-1f) {
            m = hadd(m, m);
            e = e - 1;
        }
        const float s = hdiv(hsub(m, 1.0f), hadd(m, 1.0f));
        const float s2 = hmul(s, s);
        float q = 0x1.3b13b2p-4f;  // 1/13
        q = hadd(hmul(q, s2), 0x1.745d18p-4f);
        q = hadd(hmul(q, s2), 0x1.c71c72p-4f);
        q = hadd(hmul(q, s2), 0x1.24924ap-3f);
        q = hadd(hmul(q, s2), 0x1.99999ap-3f);
        q = hadd(hmul(q, s2), 0x1.555556p-2f);
        q = hadd(hmul(q, s2), 1.0f);
        const float lg = hadd(hmul((float)e, 0x1.62e43p-1f), hmul(hadd(s, s), q));
        r = hmul(0.5f, lg);
    }
    return p < 0.0f ? -r : r;
}

// misc area of a slot
struct Misc {
    int red[32];
    long long bcast[2];
    int ints[8];
    unsigned long long okd, okit;  // converged decodes of this group and their iterations
    int K[2];                      // iteration limit of each half's candidate (two-codeword kernels)
    uint16_t seg[kMaxNb + 2];
};

// ---------------------------------------------------------------------------
// one decode
// ---------------------------------------------------------------------------
template <class Dec, int DCMAX, bool QC>
struct Decoder {
    using msg = typename Dec::msg;
    using post = typename Dec::post;
    using lv = typename Dec::lv;

    const DevCode &g;
    const SGraph &sg;
    const Grp &gp;
    const DecodeParams &dp;
    post *P;
    msg *R;

    // check pass: returns (group total) unsatisfied checks of x = [P < 0];
    // if writeR, also replaces R by the next check-to-variable messages.
    __device__ __forceinline__ int check_pass(bool first, bool writeR) const {
        int unsat = 0;
        const int Z = g.Z;
        if (QC) {
            int i = gp.gt / Z, r = gp.gt - i * Z;
            for (int c = gp.gt; c < g.m; c += gp.T) {
                const int deg = sg.rdeg[i];
                const int e0 = sg.reoff[i] + r;
                const int32_t *rjz = sg.rjz + i * g.dc_max;
                const int16_t *rs = sg.rs + i * g.dc_max;
                unsat += check_node(first, writeR, deg, e0, Z, [&](int p) {
                    return rjz[p] + wrapZ(r + rs[p], Z);
                });
                r += gp.T;
                while (r >= Z) { r -= Z; i++; }
            }
        } else {
            for (int c = gp.gt; c < g.m; c += gp.T) {
                const int e0 = sg.c_ptr[c];
                const int deg = sg.c_ptr[c + 1] - e0;
                // message (c, p) lives at p*m + c (consecutive lanes, consecutive words)
                unsat += check_node(first, writeR, deg, c, g.m, [&](int p) { return (int)sg.c_vn[e0 + p]; });
            }
        }
        return gp.sum(unsat);
    }

    template <class NB>
    __device__ __forceinline__ int check_node(bool first, bool writeR, int deg, int e0, int estride,
                                              NB nb) const {
        if constexpr (!Dec::kFloat) {
            const int sat = dp.sat;
            int m1 = sat, m2 = sat, sgn = 0, par = 0;
            int a[DCMAX];
#pragma unroll
            for (int p = 0; p < DCMAX; p++) {
                if (p < deg) {
                    const int v = nb(p);
                    const int Pv = (int)P[v];
                    const int ro = first ? 0 : (int)R[e0 + p * estride];
                    par ^= Pv;
                    const int q = clampi(Pv - ro, -sat, sat);
                    sgn |= (int)((unsigned)q >> 31) << p;
                    const int aa = abs(q);
                    a[p] = aa;
                    m2 = min(m2, max(m1, aa));
                    m1 = min(m1, aa);
                }
            }
            if (writeR) {
                const int o1 = (dp.alpha_num * m1) >> dp.alpha_shift;
                const int o2 = (dp.alpha_num * m2) >> dp.alpha_shift;
                const int tot = __popc(sgn) & 1;
#pragma unroll
                for (int p = 0; p < DCMAX; p++) {
                    if (p < deg) {
                        const int mag = a[p] == m1 ? o2 : o1;
                        const int neg = tot ^ ((sgn >> p) & 1);
                        R[e0 + p * estride] = (msg)(neg ? -mag : mag);
                    }
                }
            }
            return par < 0;
        } else {
            const float clip = dp.spa_clip;
            float t[DCMAX];
            int par = 0;
#pragma unroll
            for (int p = 0; p < DCMAX; p++) {
                if (p < deg) {
                    const int v = nb(p);
                    const float Pv = (float)P[v];
                    const float ro = first ? 0.0f : (float)R[e0 + p * estride];
                    par ^= Pv < 0.0f;
                    const float q = clampf_(__fsub_rn(Pv, ro), -clip, clip);
                    t[p] = spa_tanhf(__fmul_rn(q, 0.5f));
                }
            }
            if (writeR) {
#pragma unroll
                for (int p = 0; p < DCMAX; p++) {
                    if (p < deg) {
                        float prod = 1.0f;
#pragma unroll
                        for (int p2 = 0; p2 < DCMAX; p2++)
                            if (p2 < deg && p2 != p) prod = __fmul_rn(prod, t[p2]);
                        float rr;
                        if (fabsf(prod) >= 1.0f) rr = prod > 0.0f ? clip : -clip;
                        else rr = __fmul_rn(2.0f, spa_atanhf(prod));
                        R[e0 + p * estride] = (msg)clampf_(rr, -clip, clip);
                    }
                }
            }
            return par;
        }
    }

    // posterior of variable node v with channel value L
    __device__ __forceinline__ lv posterior(int v, lv L) const {
        lv acc = L;
        if (QC) {
            const int j = v / g.Z, k = v - j * g.Z;
            const int deg = sg.cdeg[j];
#pragma unroll 4
            for (int t = 0; t < deg; t++) {
                const int idx = j * g.dv_max + t;
                acc = acc + (lv)R[sg.ceoff[idx] + wrapZneg(k - sg.cs[idx], g.Z)];
            }
        } else {
            const int t0 = sg.v_ptr[v], t1 = sg.v_ptr[v + 1];
            for (int t = t0; t < t1; t++) acc = acc + (lv)R[sg.v_edge[t]];
        }
        return acc;
    }

    __device__ __forceinline__ void vn_pass(lv Lbase) const {
        if (QC) {
            const int Z = g.Z;
            int j = gp.gt / Z, k = gp.gt - j * Z;
            for (int v = gp.gt; v < g.n; v += gp.T) {
                const int deg = sg.cdeg[j];
                lv acc = Lbase;
#pragma unroll 4
                for (int t = 0; t < deg; t++) {
                    const int idx = j * g.dv_max + t;
                    acc = acc + (lv)R[sg.ceoff[idx] + wrapZneg(k - sg.cs[idx], Z)];
                }
                P[v] = (post)acc;
                k += gp.T;
                while (k >= Z) { k -= Z; j++; }
            }
        } else {
            for (int v = gp.gt; v < g.n; v += gp.T) {
                const int t0 = sg.v_ptr[v], t1 = sg.v_ptr[v + 1];
                lv acc = Lbase;
                for (int t = t0; t < t1; t++) acc = acc + (lv)R[sg.v_edge[t]];
                P[v] = (post)acc;
            }
        }
    }

    __device__ __forceinline__ void save_x(uint32_t *xw) const {
        for (int base = 0; base < g.n; base += gp.T) {
            const int v = base + gp.gt;
            const bool bit = v < g.n && P[v] < (post)0;
            const unsigned w = __ballot_sync(0xffffffffu, bit);
            const int wi = (base >> 5) + gp.gw;
            if (gp.lane == 0 && (wi << 5) < g.n) xw[wi] = w;
        }
    }

    // Returns true if the decode failed (x_{K_last} != 0); xbest receives x*.
    // K: the iteration limit of this candidate.
    __device__ bool run(const int *I, int nI, lv Lbase, lv Limp, uint32_t *xbest, int &kl, int K) const {
        if (!(Limp < (lv)0)) {  // x_0 = 0: u_0 = 0, success at iteration 0
            kl = 0;
            return false;
        }
        for (int v = gp.gt; v < g.n; v += gp.T) P[v] = (post)Lbase;
        gp.sync();
        if (gp.gt < nI) P[I[gp.gt]] = (post)Limp;
        gp.sync();
        int ubest = 0x7fffffff, u = 0, k = 0;
        bool first = true;
        while (true) {
            u = check_pass(first, k < K);  // u = u_k; R <- R_{k+1}
            first = false;
            if (k >= g.wstart && u < ubest) {
                ubest = u;
                save_x(xbest);
            }
            if (u == 0 || k == K) break;
            vn_pass(Lbase);  // P <- P_{k+1}
            gp.sync();
            if (gp.gt < nI) P[I[gp.gt]] = (post)posterior(I[gp.gt], Limp);
            gp.sync();
            k++;
        }
        kl = k;
        if (k < g.wstart) save_x(xbest);
        int neg = 0;
        if (u == 0)
            for (int v = gp.gt; v < g.n; v += gp.T) neg |= P[v] < (post)0;
        const int any = gp.sum(neg);
        return u != 0 || any != 0;
    }
};

// Iteration limit of candidate idx: K, or its cycle-density budget.
__device__ __forceinline__ int cand_limit(const DecodeParams &dp, const EnumBuffers &b, long long idx) {
    return b.cand_K ? (int)b.cand_K[idx] : dp.K;
}

// ---------------------------------------------------------------------------
// sieving: Tree(), TS(), (a,b)
// ---------------------------------------------------------------------------
template <bool QC>
struct Sieve {
    const DevCode &g;
    const SGraph &sg;
    const Grp &gp;

    __device__ __forceinline__ int vn_check_s(int v, int t) const {
        if (QC) {
            const int j = v / g.Z, k = v - j * g.Z;
            const int idx = j * g.dv_max + t;
            return sg.ciz[idx] + wrapZneg(k - sg.cs[idx], g.Z);
        }
        return g.v_chk[sg.v_ptr[v] + t];
    }
    __device__ __forceinline__ int vn_deg_s(int v) const {
        if (QC) return sg.cdeg[v / g.Z];
        return sg.v_ptr[v + 1] - sg.v_ptr[v];
    }
    __device__ __forceinline__ static bool bit(const uint32_t *S, int v) { return (S[v >> 5] >> (v & 31)) & 1u; }

    // deg[c] = |N(c) n S|
    __device__ void count_deg(const uint32_t *S, int *deg) const {
        for (int c = gp.gt; c < g.m; c += gp.T) {
            int cnt = 0;
            if (QC) {
                const int i = c / g.Z, r = c - i * g.Z;
                const int d = sg.rdeg[i];
                for (int p = 0; p < d; p++) {
                    const int idx = i * g.dc_max + p;
                    cnt += bit(S, sg.rjz[idx] + wrapZ(r + sg.rs[idx], g.Z));
                }
            } else {
                const int e0 = sg.c_ptr[c], e1 = sg.c_ptr[c + 1];
                for (int e = e0; e < e1; e++) cnt += bit(S, sg.c_vn[e]);
            }
            deg[c] = cnt;
        }
    }

    // Tree(S): delete variable nodes with fewer than two checks of degree >= 2
    // until none is left (the 2-core of the induced bipartite graph).
    __device__ void peel(uint32_t *S, int *deg) const {
        while (true) {
            int changed = 0;
            for (int base = 0; base < g.n; base += gp.T) {
                const int v = base + gp.gt;
                bool rm = false;
                if (v < g.n && bit(S, v)) {
                    const int d = vn_deg_s(v);
                    int live = 0;
                    for (int t = 0; t < d; t++) live += deg[vn_check_s(v, t)] >= 2;
                    rm = live < 2;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, rm);
                const int wi = (base >> 5) + gp.gw;
                if (gp.lane == 0 && mask) S[wi] &= ~mask;
                if (rm) {
                    const int d = vn_deg_s(v);
                    for (int t = 0; t < d; t++) atomicSub(&deg[vn_check_s(v, t)], 1);
                }
                changed |= mask != 0;
            }
            gp.sync();
            if (!gp.sum(changed)) break;
        }
    }

    // S <- S u {v not in S : at least two checks of v touch S} (deg = |N(c) n S|)
    __device__ void closure(uint32_t *S, const int *deg) const {
        for (int base = 0; base < g.n; base += gp.T) {
            const int v = base + gp.gt;
            bool add = false;
            if (v < g.n && !bit(S, v)) {
                const int d = vn_deg_s(v);
                int k = 0;
                for (int t = 0; t < d; t++) k += deg[vn_check_s(v, t)] >= 1;
                add = k >= 2;
            }
            const unsigned mask = __ballot_sync(0xffffffffu, add);
            const int wi = (base >> 5) + gp.gw;
            if (gp.lane == 0 && mask) S[wi] |= mask;
        }
    }

    __device__ int popcount(const uint32_t *S) const {
        const int nw = (g.n + 31) >> 5;
        int c = 0;
        for (int w = gp.gt; w < nw; w += gp.T) c += __popc(S[w]);
        return gp.sum(c);
    }

    // X = xk u I into S, and deg for it
    __device__ void load_x(uint32_t *S, const uint32_t *xk, const int *I, int nI, int *deg) const {
        const int nw = (g.n + 31) >> 5;
        for (int w = gp.gt; w < nw; w += gp.T) S[w] = xk[w];
        gp.sync();
        if (gp.gt < nI) atomicOr(&S[I[gp.gt] >> 5], 1u << (I[gp.gt] & 31));
        gp.sync();
        count_deg(S, deg);
        gp.sync();
    }

    // Returns the sieve used (1: S1 = Tree(X), 2: S2 = Tree(TS(X)), 0: both
    // empty); S holds T and deg[c] = |N(c) n T| on return.
    __device__ int run(uint32_t *S, const uint32_t *xk, const int *I, int nI, int *deg, int &a) const {
        load_x(S, xk, I, nI, deg);
        peel(S, deg);
        a = popcount(S);
        if (a > 0) return 1;
        load_x(S, xk, I, nI, deg);
        closure(S, deg);
        gp.sync();
        count_deg(S, deg);
        gp.sync();
        peel(S, deg);
        a = popcount(S);
        return a > 0 ? 2 : 0;
    }

    // b = checks of odd degree in T, elementary = every check degree <= 2
    __device__ void classify(const int *deg, int &b, int &elem) const {
        int odd = 0, big = 0;
        for (int c = gp.gt; c < g.m; c += gp.T) {
            odd += deg[c] & 1;
            big |= deg[c] > 2;
        }
        b = gp.sum(odd);
        elem = gp.sum(big) == 0;
    }
};

// ---------------------------------------------------------------------------
// canonical key, orbit, hash and insert (warp 0 of the group)
// ---------------------------------------------------------------------------
struct Cursor {
    int seg, t, w, st, c, jz;
};

__device__ __forceinline__ void cur_enter(Cursor &cu, int seg, const uint16_t *L, const uint16_t *segs,
                                          int Z, int s) {
    cu.seg = seg;
    cu.st = segs[seg];
    cu.c = segs[seg + 1] - cu.st;
    cu.t = 0;
    cu.jz = (L[cu.st] / Z) * Z;
    int w = cu.c;
    for (int x = 0; x < cu.c; x++)
        if ((int)L[cu.st + x] - cu.jz >= Z - s) { w = x; break; }
    cu.w = w;
}
__device__ __forceinline__ int cur_elem(const Cursor &cu, const uint16_t *L, int Z, int s) {
    int idx = cu.w + cu.t;
    if (idx >= cu.c) idx -= cu.c;
    int k = (int)L[cu.st + idx] - cu.jz + s;
    if (k >= Z) k -= Z;
    return cu.jz + k;
}

// Ordered list of the set bits of S (warp 0), returns count.
__device__ int list_bits(const uint32_t *S, int n, uint16_t *list, int lane) {
    const int nw = (n + 31) >> 5;
    int pos = 0;
    for (int base = 0; base < nw; base += 32) {
        const int w = base + lane;
        uint32_t x = w < nw ? S[w] : 0u;
        const int c = __popc(x);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        int off = pos + incl - c;
        while (x) {
            const int b = __ffs(x) - 1;
            x &= x - 1;
            list[off++] = (uint16_t)(w * 32 + b);
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    return pos;
}

// Canonical key (QC: smallest sorted tuple over the shifts moving a member
// to k = 0; CSR: the sorted set) into key[], returns the orbit size.
__device__ int canon_key(const DevCode &g, const uint16_t *L, int a, const uint32_t *S, uint16_t *key,
                         uint16_t *segs, int lane) {
    if (g.kind != TSX_CODE_QC) {
        for (int i = lane; i < a; i += 32) key[i] = L[i];
        __syncwarp();
        return 1;
    }
    const int Z = g.Z;
    // segments of equal column block
    int nseg = 0;
    for (int base = 0; base < a; base += 32) {
        const int i = base + lane;
        const bool mk = i < a && (i == 0 || L[i] / Z != L[i - 1] / Z);
        const unsigned mask = __ballot_sync(0xffffffffu, mk);
        if (mk) segs[nseg + __popc(mask & ((1u << lane) - 1))] = (uint16_t)i;
        nseg += __popc(mask);
    }
    if (lane == 0) segs[nseg] = (uint16_t)a;
    __syncwarp();
    // stabilizer: shifts sigma = k(L[i]) - k(L[0]) of segment-0 members
    // with T + sigma = T
    const int c0 = segs[1];
    const int k0 = L[0] % Z;
    int stab = 0;
    for (int base = 0; base < c0; base += 32) {
        const int i = base + lane;
        bool ok = i < c0;
        if (ok) {
            const int sig = (int)L[i] % Z - k0;  // >= 0: same block, ascending
            for (int x = 0; x < a && ok; x++) {
                const int v = L[x];
                const int j = v / Z;
                int k = v - j * Z + sig;
                if (k >= Z) k -= Z;
                const int u = j * Z + k;
                ok = (S[u >> 5] >> (u & 31)) & 1u;
            }
        }
        stab += __popc(__ballot_sync(0xffffffffu, ok));
    }
    // tournament over the candidate shifts s_i = -k(L[i]) mod Z
    int best_s = (Z - k0) % Z;
    for (int cs0 = 1; cs0 < a; cs0 += 31) {
        int s;
        bool active;
        if (lane == 0) {
            s = best_s;
            active = true;
        } else {
            const int i = cs0 + lane - 1;
            active = i < a;
            s = active ? (Z - (int)L[i] % Z) % Z : 0;
        }
        Cursor cu;
        cur_enter(cu, 0, L, segs, Z, s);
        for (int pos = 0; pos < a; pos++) {
            const int e = cur_elem(cu, L, Z, s);
            const int mn = __reduce_min_sync(0xffffffffu, active ? e : 0x7fffffff);
            active = active && e == mn;
            if (__popc(__ballot_sync(0xffffffffu, active)) <= 1) break;
            if (++cu.t == cu.c && cu.seg + 1 < nseg) cur_enter(cu, cu.seg + 1, L, segs, Z, s);
        }
        const unsigned am = __ballot_sync(0xffffffffu, active);
        best_s = __shfl_sync(0xffffffffu, s, __ffs(am) - 1);
    }
    // write the key for best_s
    for (int pos = lane; pos < a; pos += 32) {
        int seg = 0;
        while (seg + 1 < nseg && segs[seg + 1] <= pos) seg++;
        Cursor cu;
        cur_enter(cu, seg, L, segs, Z, best_s);
        cu.t = pos - cu.st;
        key[pos] = (uint16_t)cur_elem(cu, L, Z, best_s);
    }
    __syncwarp();
    return Z / stab;
}

__device__ unsigned long long key_hash(const uint16_t *key, int a, int lane) {
    unsigned long long h = 0;
    for (int i = lane; i < a; i += 32) h += mix64(((unsigned long long)i << 32) | key[i]);
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    return h + mix64(0xabcdef0000000000ull + (unsigned long long)a);
}

// Space reserved at pool offset off for a key of a nodes that another
// insert of the same key made unnecessary: taken back if nothing was
// reserved after it, else counted as leaked.
__device__ __forceinline__ void pool_giveback(const EnumBuffers &b, long long off, int a) {
    const unsigned long long len = (unsigned long long)(kPoolHdr + a);
    const unsigned long long top = (unsigned long long)(off - 1);  // pool_top before the reservation
    if (atomicCAS(&b.ctr->pool_top, top + len, top) != top + len) atomicAdd(&b.ctr->pool_leaked, len);
}

// Insert / find the key; returns the table slot, -1 on a full table, -2 on
// a pool overflow.  Warp-collective.  The header's flags word ends as the OR
// of the flags of every insert of the key (independent of their order).
__device__ long long ts_insert(const EnumBuffers &b, const uint16_t *key, int a, int bb, int orbit,
                               int flags, int lane) {
    const unsigned long long h = key_hash(key, a, lane);
    const unsigned long long hhi = (h >> 32) << 32;
    unsigned long long slot = h & b.cap_mask;
    long long my_off = -1;
    for (unsigned long long probe = 0; probe <= b.cap_mask; probe++) {
        unsigned long long tag = 0;
        if (lane == 0) tag = *((volatile unsigned long long *)&b.tags[slot]);
        tag = __shfl_sync(0xffffffffu, tag, 0);
        if (tag == 0) {
            if (my_off < 0) {
                long long off = 0;
                // word 0 of the pool is never used, so a tag is never 0
                if (lane == 0) off = 1 + (long long)atomicAdd(&b.ctr->pool_top, (unsigned long long)(kPoolHdr + a));
                off = __shfl_sync(0xffffffffu, off, 0);
                if ((unsigned long long)(off + kPoolHdr + a) > b.pool_cap + 1) {
                    if (lane == 0) atomicOr(&b.ctr->err, kErrPoolOverflow);
                    return -2;
                }
                if (lane == 0) {
                    b.pool[off] = a;
                    b.pool[off + 1] = bb;
                    b.pool[off + 2] = orbit;
                    b.pool[off + 3] = flags;
                }
                for (int i = lane; i < a; i += 32) b.pool[off + kPoolHdr + i] = key[i];
                __threadfence();
                __syncwarp();
                my_off = off;
            }
            unsigned long long old = 0;
            if (lane == 0) old = atomicCAS(&b.tags[slot], 0ull, hhi | (unsigned long long)my_off);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == 0) return (long long)slot;
            tag = old;
        }
        if ((tag & 0xffffffff00000000ull) == hhi) {
            __threadfence();
            const long long off = (long long)(tag & 0xffffffffull);
            bool eq = __ldcg(&b.pool[off]) == a;
            if (eq)
                for (int i = lane; i < a && eq; i += 32) eq = __ldcg(&b.pool[off + kPoolHdr + i]) == (int)key[i];
            if (__all_sync(0xffffffffu, eq)) {
                // the sieve bits of a set are the union over every candidate that reached it
                if (lane == 0) {
                    atomicOr(&b.pool[off + 3], flags);
                    if (my_off >= 0) pool_giveback(b, my_off, a);
                }
                return (long long)slot;
            }
        }
        slot = (slot + 1) & b.cap_mask;
    }
    if (lane == 0) {
        atomicOr(&b.ctr->err, kErrTableFull);
        if (my_off >= 0) pool_giveback(b, my_off, a);
    }
    return -1;
}

// ---------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------
template <class Dec, int DCMAX, bool QC>
__device__ __forceinline__ void scalar_run(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b,
                                           const SlotLayout &lay, int G, const SGraph &sg, unsigned char *smem,
                                           int grp) {
    using lv = typename Dec::lv;
    using post = typename Dec::post;
    using msg = typename Dec::msg;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    post *P = (post *)(slot + lay.p_off);
    msg *R = (msg *)(slot + lay.r_off);
    uint32_t *xa = (uint32_t *)(slot + lay.xa_off);
    uint32_t *xb = (uint32_t *)(slot + lay.xb_off);

    Decoder<Dec, DCMAX, QC> dec{g, sg, gp, dp, P, R};

    const long long total = (long long)b.ctr->n_cand_total;
    const long long end = b.cand_end < 0 || b.cand_end > total ? total : b.cand_end;
    long long my_dec = 0, my_it = 0, my_eu = 0, my_ok = 0, my_okit = 0;

    lv Lbase;
    if constexpr (Dec::kFloat) Lbase = (lv)clampf_((float)dp.base_llr / 8.0f, -dp.spa_clip, dp.spa_clip);
    else Lbase = (lv)clampi(dp.base_llr, -dp.sat, dp.sat);

    while (true) {
        if (gp.gt == 0) misc->bcast[0] = (long long)atomicAdd(b.queue, 1ull);
        gp.sync();
        const long long idx = b.cand_begin + misc->bcast[0];
        gp.sync();
        if (idx >= end) break;
        const int4 I4 = b.cands[idx];
        int I[4] = {I4.x, I4.y, I4.z, I4.w};
        const int nI = (I4.x >= 0) + (I4.y >= 0) + (I4.z >= 0) + (I4.w >= 0);

        uint32_t *xcur = xa, *xkeep = xb;
        int ndec = 0, nit = 0, kl = 0;
        bool failed = false;
        int thr = -1;
        float thr_f = -1.0f;
        const int Kc = cand_limit(dp, b, idx);
        if constexpr (!Dec::kFloat) {
            int lo = 0, hi = (1 << dp.amp_steps) - 1;
            bool f = dec.run(I, nI, Lbase, (lv)clampi(dp.base_llr - hi, -dp.sat, dp.sat), xcur, kl, Kc);
            ndec++;
            nit += kl;
            if (!f) { my_ok++; my_okit += kl; }
            if (f) {
                failed = true;
                uint32_t *t = xcur; xcur = xkeep; xkeep = t;
                for (int st = 0; st < dp.amp_steps && hi - lo > 1; st++) {
                    const int mid = (lo + hi) >> 1;
                    f = dec.run(I, nI, Lbase, (lv)clampi(dp.base_llr - mid, -dp.sat, dp.sat), xcur, kl, Kc);
                    ndec++;
                    nit += kl;
                    if (!f) { my_ok++; my_okit += kl; }
                    if (f) {
                        hi = mid;
                        uint32_t *t2 = xcur; xcur = xkeep; xkeep = t2;
                    } else {
                        lo = mid;
                    }
                }
                thr = hi;
            }
        } else {
            float lo = 0.0f, hi = 1.0f;
            const float basef = (float)dp.base_llr / 8.0f;
            auto limp = [&](float eps) {
                return (lv)clampf_(__fsub_rn(basef, __fmul_rn(eps, dp.spa_amax)), -dp.spa_clip, dp.spa_clip);
            };
            bool f = dec.run(I, nI, Lbase, limp(hi), xcur, kl, Kc);
            ndec++;
            nit += kl;
            if (!f) { my_ok++; my_okit += kl; }
            if (f) {
                failed = true;
                uint32_t *t = xcur; xcur = xkeep; xkeep = t;
                for (int st = 0; st < dp.amp_steps; st++) {
                    const float mid = __fmul_rn(0.5f, __fadd_rn(lo, hi));
                    f = dec.run(I, nI, Lbase, limp(mid), xcur, kl, Kc);
                    ndec++;
                    nit += kl;
                    if (!f) { my_ok++; my_okit += kl; }
                    if (f) {
                        hi = mid;
                        uint32_t *t2 = xcur; xcur = xkeep; xkeep = t2;
                    } else {
                        lo = mid;
                    }
                }
                thr_f = hi;
            }
        }
        my_dec += ndec;
        my_it += nit;
        my_eu += (long long)nit * g.E;

        // records and the failing decode's x* for the sieve kernel
        gp.sync();
        const long long o = idx - b.rec_base;
        if (failed) {
            uint32_t *dst = b.xstar + o * (long long)b.nw;
            for (int w = gp.gt; w < b.nw; w += gp.T) dst[w] = xkeep[w];
        }
        if (gp.gt == 0) {
            b.c_thr[o] = thr;
            b.c_thr_f[o] = thr_f;
            b.c_slot[o] = -1;
            b.c_flags[o] = 0;
            b.c_decodes[o] = ndec;
            b.c_iters[o] = nit;
        }
        gp.sync();
    }
    if (gp.gt == 0) {
        atomicAdd(&b.ctr->decodes, (unsigned long long)my_dec);
        atomicAdd(&b.ctr->iterations, (unsigned long long)my_it);
        atomicAdd(&b.ctr->edge_updates, (unsigned long long)my_eu);
        atomicAdd(&b.ctr->ok_decodes, (unsigned long long)my_ok);
        atomicAdd(&b.ctr->ok_iters, (unsigned long long)my_okit);
    }
}

template <class Dec, int DCMAX, bool QC>
__global__ void __launch_bounds__(512, 1) enum_kernel(DevCode g, DecodeParams dp, EnumBuffers b,
                                                    SlotLayout lay, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem);
    __syncthreads();
    scalar_run<Dec, DCMAX, QC>(g, dp, b, lay, G, sg, smem, (threadIdx.x >> 5) / G);
}

// ---------------------------------------------------------------------------
// the sieve kernel: one warp per failing candidate
// ---------------------------------------------------------------------------
template <bool QC>
__global__ void __launch_bounds__(512) sieve_kernel(DevCode g, EnumBuffers b, SlotLayout lay, int is_float) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *slot = smem + lay.tables_bytes + warp * lay.slot_bytes;
    Misc *misc = (Misc *)(slot + lay.misc_off);
    Grp gp;
    gp.G = 1;
    gp.T = 32;
    gp.gw = 0;
    gp.gt = lane;
    gp.lane = lane;
    gp.bar = 1;
    gp.red = misc->red;
    int *deg = (int *)(slot + lay.r_off);
    uint16_t *key = (uint16_t *)(slot + lay.r_off);
    uint16_t *L = (uint16_t *)(slot + lay.p_off);
    uint32_t *S = (uint32_t *)(slot + lay.xa_off);
    Sieve<QC> sv{g, sg, gp};

    const long long total = (long long)b.ctr->n_cand_total;
    const long long end = b.cand_end < 0 || b.cand_end > total ? total : b.cand_end;
    const long long n = end - b.cand_begin;
    long long my_acyc = 0;
    while (true) {
        long long o = 0;
        if (lane == 0) o = (long long)atomicAdd(&b.ctr->next_sieve, 1ull);
        o = __shfl_sync(0xffffffffu, o, 0);
        if (o >= n) break;
        const bool failed = is_float ? b.c_thr_f[o] >= 0.0f : b.c_thr[o] >= 0;
        if (!failed) continue;
        const int4 I4 = b.cands[b.cand_begin + o];
        int I[4] = {I4.x, I4.y, I4.z, I4.w};
        const int nI = (I4.x >= 0) + (I4.y >= 0) + (I4.z >= 0) + (I4.w >= 0);
        const uint32_t *xk = b.xstar + o * (long long)b.nw;
        int a = 0;
        const int which = sv.run(S, xk, I, nI, deg, a);
        int flags = which;
        long long tslot = -1;
        if (which == 0) {
            flags |= kFlagAcyclic;
            my_acyc++;
        } else {
            int bb, elem;
            sv.classify(deg, bb, elem);
            __syncwarp();
            list_bits(S, g.n, L, lane);
            const int orbit = canon_key(g, L, a, S, key, misc->seg, lane);
            const int thr_ord = is_float ? f2ord(b.c_thr_f[o]) : b.c_thr[o];
            tslot = ts_insert(b, key, a, bb, orbit, elem | (which << 1), lane);
            if (tslot >= 0 && lane == 0) {
                atomicMin(&b.t_thr[tslot], thr_ord);
                atomicAdd(&b.t_count[tslot], 1);
            }
            if (tslot == -2) flags |= kFlagOverflow;
        }
        if (lane == 0) {
            b.c_slot[o] = (int)(tslot >= 0 ? tslot : -1);
            b.c_flags[o] = flags;
        }
        __syncwarp();
    }
    if (lane == 0 && my_acyc) atomicAdd(&b.ctr->acyclic, (unsigned long long)my_acyc);
}


// launches one instantiation of a persistent kernel with every CTA resident
template <class K, class... Args>
cudaError_t launch_persistent(K k, const LaunchShape &sh, cudaStream_t st, Args... args) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, sh.smem_bytes);
    if (e != cudaSuccess) return e;
    const int threads = sh.groups * sh.G * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, sh.smem_bytes);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    if (sh.per_sm_req > 0 && sh.per_sm_req < occ) occ = sh.per_sm_req;
    k<<<occ * sh.num_sms, threads, sh.smem_bytes, st>>>(args...);
    return cudaGetLastError();
}

// the scalar kernel (one codeword per group)
template <class Dec>
cudaError_t launch_scalar(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                          cudaStream_t st) {
    const bool qc = g.kind == TSX_CODE_QC;
    if (g.dc_max <= 8)
        return qc ? launch_persistent(enum_kernel<Dec, 8, true>, sh, st, g, dp, b, sh.lay, sh.G)
                  : launch_persistent(enum_kernel<Dec, 8, false>, sh, st, g, dp, b, sh.lay, sh.G);
    return qc ? launch_persistent(enum_kernel<Dec, 32, true>, sh, st, g, dp, b, sh.lay, sh.G)
              : launch_persistent(enum_kernel<Dec, 32, false>, sh, st, g, dp, b, sh.lay, sh.G);
}

}  // namespace
}  // namespace tsx
