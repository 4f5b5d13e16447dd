// decode_pair.cuh -- the fixed-point min-sum impulse decoder, two codewords
// per lane.
//
// A group of G warps owns a pair of codeword slots ("halves" 0 and 1) and
// runs two independent candidates at once: every shared-memory word holds
// the same message or posterior of both codewords, one per 16-bit half, and
// the two halves follow their own bisection and decode schedules (a half
// whose decode ends starts its next decode at once; the other keeps going).
//
// Biased representation (so that one 32-bit add or subtract updates both
// halves without a carry or borrow crossing between them, and signs and
// equalities are single bits):
//   message   R' = r + B                     B = 1024 (int16) / 128 (int8)
//   posterior P' = P + beta                  beta = 0x8000
//   channel   L'(v) = L_v + beta - dv(v) B   so P' = L' + sum_c R'
//   extrinsic d = P' - R' + B = q + beta     (one three-input add): bit 15 of each half is
//                                           [q >= 0], the sign of clamp(q); the clamp itself
//                                           is not applied (edge_da says why it changes nothing)
//   magnitude a = max(d, 2 beta - d) = |q| + beta   (2 beta - x = ~x + 1 per half)
// Every intermediate stays inside [0, 0xFFFF] per half for rmax <= B and
// (dv + 2) sat <= beta - B, which the launcher checks; both halves always
// hold values of a valid decode (an idle half keeps decoding its last input)
// so that neither can carry into the other.  The arithmetic is the same
// min-sum as the scalar decoder: r = sgn * ((alpha_num * min) >> alpha_shift)
// over the other edges of the check, P = L + sum r, q = clamp(P - r).
//
// No variable-node pass: each check adds its new messages into the next
// posterior buffer with shared-memory atomic adds (exact and order-free on
// the biased words); that buffer starts at L' with the impulse values in it.
// For QC codes whose two buffers do not fit a CTA, the variable-node-pass
// form (VN) keeps one buffer and rebuilds it from the messages after each
// check pass; it gives the same words.
//
// The first check pass of a decode reads the zero message B in its half; a
// check pass in which no half starts a decode skips that masking.
#pragma once
#include "decode_impl.cuh"

namespace tsx {
namespace {

__device__ __forceinline__ unsigned vmaxu2(unsigned a, unsigned b) {
    unsigned d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ unsigned vminu2(unsigned a, unsigned b) {
    unsigned d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ unsigned prmt(unsigned a, unsigned b, unsigned sel) {
    unsigned d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}
// 0xFFFF in each half whose bit 15 is set, else 0
__device__ __forceinline__ unsigned spread15(unsigned x) { return prmt(x, x, 0xBB99u); }
__device__ __forceinline__ void red_add(unsigned char *addr, unsigned v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(addr)), "r"(v)
                 : "memory");
}

constexpr unsigned kBeta = 0x8000u;

struct PairConst {
    unsigned B2, BS2, BETA2, amask2;
    unsigned BAN2;  // BETA2 * alpha_num: (m - beta) an = m an - BAN2 (mod 2^32)
    int B, sat, an, as;
};

// per-half schedule state (uniform across the group)
struct Half {
    long long idx;  // candidate (absolute index), -1: idle
    int I0, I1, I2, I3, nI;
    int lo, hi, st, phase;  // bisection
    int thr, ndec, nit;
    int failed;
    int Limp;  // channel LLR of the impulse nodes in the current decode
    int k, ubest;
    int first;  // current decode has run no check pass yet
    int cur;    // x buffer of the current decode (0/1); keep = cur ^ 1
    __device__ __forceinline__ int Ik(int t) const { return t == 0 ? I0 : t == 1 ? I1 : t == 2 ? I2 : I3; }
};

// VN: the variable-node-pass form (QC codes): one posterior buffer, rebuilt
// after each check pass from the stored messages, instead of the
// accumulating second buffer -- 4 bytes per node less, for codes whose
// two-buffer layout does not fit a CTA.
// FLAT (QC, accumulating form): the check pass runs over all row blocks at
// once, as the VN form does, so that a group may be wider than Z rows.
template <bool QC, int DC, bool EXACT, bool I8, bool VN = false, bool FLAT = false>
struct PairDecoder {
    static constexpr int RSZ = I8 ? 2 : 4;  // bytes of one packed message pair
    const DevCode &g;
    const SGraph &sg;
    const Grp &gp;
    const PairConst &pc;
    unsigned char *Rb;  // packed messages, RSZ bytes per edge

    __device__ __forceinline__ unsigned ldR(int byteoff) const {
        if constexpr (I8) {
            const unsigned x = *(const uint16_t *)(Rb + byteoff);
            return prmt(x, 0u, 0x4140u);  // bytes b0, b1 -> halves
        } else {
            return *(const unsigned *)(Rb + byteoff);
        }
    }
    __device__ __forceinline__ void stR(int byteoff, unsigned v) const {
        if constexpr (I8) *(uint16_t *)(Rb + byteoff) = (uint16_t)prmt(v, 0u, 0x0020u);
        else *(unsigned *)(Rb + byteoff) = v;
    }

    // an edge's incoming message; MASK: some half starts a decode in this
    // pass and reads the zero message B there (km keeps the other half, kb
    // supplies B)
    template <bool MASK>
    __device__ __forceinline__ unsigned ldy(int byteoff, unsigned km, unsigned kb) const {
        if constexpr (MASK) return (ldR(byteoff) & km) | kb;
        else return ldR(byteoff);
    }

    // One check node.  pv(p): byte offset of P'[v_p]; re(p): byte offset of
    // R'[e_p].  Reads Pc, adds the new messages into Pn.  Returns the
    // unsatisfied flags of both halves in bits 0/1.
    template <bool MASK, class PV, class RE>
    __device__ __forceinline__ int check_node(int deg, unsigned km, unsigned kb, bool writeR, const unsigned char *Pc,
                                              unsigned char *Pn, PV pv, RE re) const {
        if constexpr (DC <= 8) return check_node_regs<MASK>(deg, km, kb, writeR, Pc, Pn, pv, re);
        else return check_node_twopass<MASK>(deg, km, kb, writeR, Pc, Pn, pv, re);
    }

    // the extrinsic value of one edge without clamping: d = (P - r) + beta, which the launcher's
    // bounds keep inside each half and which has the sign of clamp(P - r),
    // and a = |P - r| + beta.  Where |P - r| > sat the clamped magnitude
    // would be sat: min1 and min2 start at sat (+ beta), so they come out
    // the same, and such an edge's output is the same too -- it is not the
    // minimum unless min1 = min2 = sat, when both outputs are equal.
    // |P - r| <= sat + (dv - 1) B < 2^15 by the launcher's bounds, so
    // a - min1 + 0x7FFF stays inside each half, as edge_out needs.
    __device__ __forceinline__ void edge_da(unsigned x, unsigned y, unsigned &d, unsigned &a) const {
        d = x - y + pc.B2;
        a = vmaxu2(d, (~d) + 0x00010001u);
    }

    // the new message of an edge from its q'', |q|, the check's min1, the
    // two output magnitudes and the sign parity of all its edges
    // (the four possible outputs B +- o1, B +- o2 are formed once per check)
    struct Outs {
        unsigned p1, n1, p2, n2;
    };
    __device__ __forceinline__ Outs outs(unsigned o1, unsigned o2) const {
        return Outs{pc.B2 + o1, pc.B2 - o1, pc.B2 + o2, pc.B2 - o2};
    }
    __device__ __forceinline__ unsigned edge_out(unsigned q, unsigned a, unsigned m1, const Outs &o,
                                                 unsigned sxk) const {
        const unsigned neg = spread15(sxk ^ q);                  // 0xFFFF: others' sign product < 0
        const unsigned ne = spread15(a - m1 + 0x7FFF7FFFu);      // 0xFFFF: |q_p| != min1
        const unsigned t1 = (o.n1 & neg) | (o.p1 & ~neg);        // +-o1
        const unsigned t2 = (o.n2 & neg) | (o.p2 & ~neg);        // +-o2
        return (t1 & ne) | (t2 & ~ne);
    }

    // small degree: the edges' q and |q| stay in registers between the passes
    template <bool MASK, class PV, class RE>
    __device__ __forceinline__ int check_node_regs(int deg, unsigned km, unsigned kb, bool writeR,
                                                   const unsigned char *Pc, unsigned char *Pn, PV pv, RE re) const {
        unsigned sp = 0, sx = 0, m1 = pc.BS2, m2 = pc.BS2;
        unsigned qs[DC], as_[DC];
        int po[DC];
#pragma unroll
        for (int p = 0; p < DC; p++) {
            if (EXACT || p < deg) {
                po[p] = pv(p);
                const unsigned x = *(const unsigned *)(Pc + po[p]);
                const unsigned y = ldy<MASK>(re(p), km, kb);
                sp ^= x;
                unsigned q, a;
                edge_da(x, y, q, a);
                sx ^= q;
                m2 = vminu2(m2, vmaxu2(m1, a));
                m1 = vminu2(m1, a);
                qs[p] = q;
                as_[p] = a;
            }
        }
        // syndrome bit of each half: sp bit 15 = parity of #(P >= 0), and
        // #(P < 0) = deg - #(P >= 0)
        const unsigned dodd = (deg & 1) ? 0x80008000u : 0u;
        const unsigned unsat = (sp ^ dodd) & 0x80008000u;
        if (writeR) {
            const unsigned o1 = ((m1 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o2 = ((m2 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const Outs oo = outs(o1, o2);
            // bit 15 of sx ^ q_p = parity of #(q >= 0) over the other edges;
            // negatives among the others = (deg - 1) - that
            const unsigned sxk = sx ^ (((deg - 1) & 1) ? 0x80008000u : 0u);
#pragma unroll
            for (int p = 0; p < DC; p++) {
                if (EXACT || p < deg) {
                    const unsigned rn = edge_out(qs[p], as_[p], m1, oo, sxk);
                    stR(re(p), rn);
                    if constexpr (!VN) red_add(Pn + po[p], rn);
                }
            }
        }
        return (int)((unsat >> 15) & 0x00010001u);
    }

    // check-regular codes (EXACT, 16-bit storage, DC even): the check's DC
    // message words are contiguous (check-major layout, 4 DC bytes a check;
    // for QC codes within each row block) and move as DC/2 8-byte accesses;
    // a warp's 8-byte accesses at a stride of 4 DC bytes = 24 bytes (DC = 6)
    // touch every bank once per half-warp.  Otherwise the same steps as
    // check_node_regs.
    template <bool MASK, class PV>
    __device__ __forceinline__ int check_node_cm(int rbyte, unsigned km, unsigned kb, bool writeR,
                                                 const unsigned char *Pc, unsigned char *Pn, PV pv) const {
        static_assert(EXACT && !I8 && DC % 2 == 0, "check-major form");
        uint2 *rw = (uint2 *)(Rb + rbyte);
        unsigned ys[DC];
#pragma unroll
        for (int t = 0; t < DC / 2; t++) {
            const uint2 w = rw[t];
            ys[2 * t] = w.x;
            ys[2 * t + 1] = w.y;
        }
        unsigned sp = 0, sx = 0, m1 = pc.BS2, m2 = pc.BS2;
        unsigned qs[DC], as_[DC];
        int po[DC];
#pragma unroll
        for (int p = 0; p < DC; p++) {
            po[p] = pv(p);
            const unsigned x = *(const unsigned *)(Pc + po[p]);
            const unsigned y = MASK ? ((ys[p] & km) | kb) : ys[p];
            sp ^= x;
            unsigned q, a;
            edge_da(x, y, q, a);
            sx ^= q;
            m2 = vminu2(m2, vmaxu2(m1, a));
            m1 = vminu2(m1, a);
            qs[p] = q;
            as_[p] = a;
        }
        const unsigned unsat = (sp ^ ((DC & 1) ? 0x80008000u : 0u)) & 0x80008000u;
        if (writeR) {
            const unsigned o1 = ((m1 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o2 = ((m2 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const Outs oo = outs(o1, o2);
            const unsigned sxk = sx ^ (((DC - 1) & 1) ? 0x80008000u : 0u);
#pragma unroll
            for (int p = 0; p < DC; p++) ys[p] = edge_out(qs[p], as_[p], m1, oo, sxk);
#pragma unroll
            for (int t = 0; t < DC / 2; t++) rw[t] = make_uint2(ys[2 * t], ys[2 * t + 1]);
#pragma unroll
            for (int p = 0; p < DC; p++)
                if constexpr (!VN) red_add(Pn + po[p], ys[p]);
        }
        return (int)((unsat >> 15) & 0x00010001u);
    }

    // large degree: the first pass leaves each edge's extrinsic word d in its
    // message slot (16-bit storage: a slot holds both halves' d), the second
    // reads it back; with 8-bit storage the second pass reloads P and
    // recomputes d
    template <bool MASK, class PV, class RE>
    __device__ __forceinline__ int check_node_twopass(int deg, unsigned km, unsigned kb, bool writeR,
                                                      const unsigned char *Pc, unsigned char *Pn, PV pv,
                                                      RE re) const {
        unsigned sp = 0, sx = 0, m1 = pc.BS2, m2 = pc.BS2;
#pragma unroll 4
        for (int p = 0; p < deg; p++) {
            const int ro = re(p);
            const unsigned x = *(const unsigned *)(Pc + pv(p));
            const unsigned y = ldy<MASK>(ro, km, kb);
            sp ^= x;
            unsigned q, a;
            edge_da(x, y, q, a);
            if constexpr (!I8)
                if (writeR) stR(ro, q);
            sx ^= q;
            m2 = vminu2(m2, vmaxu2(m1, a));
            m1 = vminu2(m1, a);
        }
        const unsigned dodd = (deg & 1) ? 0x80008000u : 0u;
        const unsigned unsat = (sp ^ dodd) & 0x80008000u;
        if (writeR) {
            const unsigned o1 = ((m1 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o2 = ((m2 * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const Outs oo = outs(o1, o2);
            const unsigned sxk = sx ^ (((deg - 1) & 1) ? 0x80008000u : 0u);
#pragma unroll 4
            for (int p = 0; p < deg; p++) {
                const int po = pv(p), ro = re(p);
                unsigned q, a;
                if constexpr (!I8) {
                    q = ldR(ro);
                    a = vmaxu2(q, (~q) + 0x00010001u);
                } else {
                    const unsigned x = *(const unsigned *)(Pc + po);
                    const unsigned y = ldy<MASK>(ro, km, kb);
                    edge_da(x, y, q, a);
                }
                const unsigned rn = edge_out(q, a, m1, oo, sxk);
                stR(ro, rn);
                if constexpr (!VN) red_add(Pn + po, rn);
            }
        }
        return (int)((unsat >> 15) & 0x00010001u);
    }

    // Two checks of one QC row block at once (rows r and r + dr, 16-bit
    // storage, large degree): the same steps as check_node_twopass for both,
    // interleaved edge by edge, so that the two dependency chains overlap and
    // each position's shift is read once for both rows.  Returns the
    // unsatisfied flags of row r in bits 0/1 and of row r + dr in bits 2/3.
    template <bool MASK>
    __device__ __forceinline__ int check_rows2(int deg, unsigned km, unsigned kb, bool writeR,
                                               const unsigned char *Pc, unsigned char *Pn, const int32_t *rjz,
                                               const int16_t *rs, int rb, int r, int dr) const {
        const int Z = g.Z;
        unsigned spA = 0, sxA = 0, m1A = pc.BS2, m2A = pc.BS2;
        unsigned spB = 0, sxB = 0, m1B = pc.BS2, m2B = pc.BS2;
        const int r2 = r + dr;
#pragma unroll 2
        for (int p = 0; p < deg; p++) {
            const int jz = rjz[p], sh = rs[p];
            const int tA = r + sh, tB = r2 + sh;
            const int poA = 4 * (jz + (int)min((unsigned)tA, (unsigned)(tA - Z)));
            const int poB = 4 * (jz + (int)min((unsigned)tB, (unsigned)(tB - Z)));
            const int roA = rb + (p * Z + r) * RSZ, roB = roA + dr * RSZ;
            const unsigned xA = *(const unsigned *)(Pc + poA), xB = *(const unsigned *)(Pc + poB);
            const unsigned yA = ldy<MASK>(roA, km, kb), yB = ldy<MASK>(roB, km, kb);
            spA ^= xA;
            spB ^= xB;
            unsigned qA, aA, qB, aB;
            edge_da(xA, yA, qA, aA);
            edge_da(xB, yB, qB, aB);
            if (writeR) {
                stR(roA, qA);
                stR(roB, qB);
            }
            sxA ^= qA;
            sxB ^= qB;
            m2A = vminu2(m2A, vmaxu2(m1A, aA));
            m1A = vminu2(m1A, aA);
            m2B = vminu2(m2B, vmaxu2(m1B, aB));
            m1B = vminu2(m1B, aB);
        }
        const unsigned dodd = (deg & 1) ? 0x80008000u : 0u;
        const unsigned unsatA = (spA ^ dodd) & 0x80008000u, unsatB = (spB ^ dodd) & 0x80008000u;
        if (writeR) {
            const unsigned o1A = ((m1A * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o2A = ((m2A * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o1B = ((m1B * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const unsigned o2B = ((m2B * (unsigned)pc.an - pc.BAN2) >> pc.as) & pc.amask2;
            const Outs ooA = outs(o1A, o2A), ooB = outs(o1B, o2B);
            const unsigned odd = ((deg - 1) & 1) ? 0x80008000u : 0u;
            const unsigned sxkA = sxA ^ odd, sxkB = sxB ^ odd;
#pragma unroll 2
            for (int p = 0; p < deg; p++) {
                const int jz = rjz[p], sh = rs[p];
                const int tA = r + sh, tB = r2 + sh;
                const int poA = 4 * (jz + (int)min((unsigned)tA, (unsigned)(tA - Z)));
                const int poB = 4 * (jz + (int)min((unsigned)tB, (unsigned)(tB - Z)));
                const int roA = rb + (p * Z + r) * RSZ, roB = roA + dr * RSZ;
                const unsigned qA = ldR(roA), qB = ldR(roB);
                const unsigned aA = vmaxu2(qA, (~qA) + 0x00010001u), aB = vmaxu2(qB, (~qB) + 0x00010001u);
                const unsigned rnA = edge_out(qA, aA, m1A, ooA, sxkA);
                const unsigned rnB = edge_out(qB, aB, m1B, ooB, sxkB);
                stR(roA, rnA);
                stR(roB, rnB);
                if constexpr (!VN) {
                    red_add(Pn + poA, rnA);
                    red_add(Pn + poB, rnB);
                }
            }
        }
        return (int)(((unsatA >> 15) & 0x00010001u) + ((unsatB >> 15) & 0x00010001u));
    }

    // check pass; returns u of half 0 in the low 16 bits and half 1 above (the
    // caller passes a group barrier before the next check pass)
    template <bool MASK>
    __device__ __forceinline__ int check_pass(unsigned km, unsigned kb, bool writeR, const unsigned *Pcur,
                                              unsigned *Pnext) const {
        int u = 0;  // unsatisfied checks: half 0 in the low 16 bits, half 1 above
        const unsigned char *Pc = (const unsigned char *)Pcur;
        unsigned char *Pn = (unsigned char *)Pnext;
        const int Z = g.Z;
        if constexpr (QC && (VN || FLAT)) {
            // all row blocks at once (check c = i Z + r), so that a group may be wider than Z rows
            const unsigned zm = Z > 1 ? 0xFFFFFFFFu / (unsigned)Z + 1u : 0u;  // c / Z = umulhi(c, zm), c < 2^16
            for (int c = gp.gt; c < g.m; c += gp.T) {
                const int i = Z > 1 ? (int)__umulhi((unsigned)c, zm) : c;
                const int r = c - i * Z;
                const int deg = sg.rdeg[i];
                const int rb = sg.reoff[i] * RSZ;
                const int32_t *rjz = sg.rjz + i * g.dc_max;
                const int16_t *rs = sg.rs + i * g.dc_max;
                u += check_node<MASK>(
                    deg, km, kb, writeR, Pc, Pn,
                    [&](int p) {
                        const int t = r + rs[p];
                        return 4 * (rjz[p] + (int)min((unsigned)t, (unsigned)(t - Z)));
                    },
                    [&](int p) { return rb + (p * Z + r) * RSZ; });
            }
        } else if constexpr (QC) {
            for (int i = 0; i < g.m_b; i++) {
                const int deg = EXACT ? DC : sg.rdeg[i];
                const int rb = sg.reoff[i] * RSZ;
                if constexpr (DC <= 8) {  // the row block's shifts in registers
                    int rjz4[DC], rsh[DC], pz[DC];
#pragma unroll
                    for (int p = 0; p < DC; p++) {
                        if (EXACT || p < deg) {
                            rjz4[p] = sg.rjz[i * g.dc_max + p] * 4;
                            rsh[p] = sg.rs[i * g.dc_max + p];
                            pz[p] = p * Z * RSZ;
                        }
                    }
                    for (int r = gp.gt; r < Z; r += gp.T) {
                        const auto pv = [&](int p) {
                            const int t = r + rsh[p];
                            return rjz4[p] + 4 * (int)min((unsigned)t, (unsigned)(t - Z));
                        };
                        if constexpr (EXACT && !I8 && DC % 2 == 0) {
                            // check-regular row blocks: messages check-major within the block
                            u += check_node_cm<MASK>(rb + r * (DC * RSZ), km, kb, writeR, Pc, Pn, pv);
                        } else {
                            u += check_node<MASK>(deg, km, kb, writeR, Pc, Pn, pv,
                                                  [&](int p) { return rb + pz[p] + r * RSZ; });
                        }
                    }
                } else {
                    const int32_t *rjz = sg.rjz + i * g.dc_max;
                    const int16_t *rs = sg.rs + i * g.dc_max;
                    int r = gp.gt;
                    if constexpr (!I8) {
                        // rows in pairs (r, r + T) while both exist
                        for (; r + gp.T < Z; r += 2 * gp.T) {
                            const int f = check_rows2<MASK>(deg, km, kb, writeR, Pc, Pn, rjz, rs, rb, r, gp.T);
                            u += f;
                        }
                    }
                    for (; r < Z; r += gp.T) {
                        const int f = check_node<MASK>(
                            deg, km, kb, writeR, Pc, Pn,
                            [&](int p) {
                                const int t = r + rs[p];
                                return 4 * (rjz[p] + (int)min((unsigned)t, (unsigned)(t - Z)));
                            },
                            [&](int p) { return rb + (p * Z + r) * RSZ; });
                        u += f;
                    }
                }
            }
        } else if constexpr (EXACT && !I8 && DC % 2 == 0) {
            // check-regular: rows of DC edges, messages check-major
            for (int c = gp.gt; c < g.m; c += gp.T) {
                const int e0 = c * DC;
                u += check_node_cm<MASK>(e0 * RSZ, km, kb, writeR, Pc, Pn,
                                         [&](int p) { return 4 * (int)sg.c_vn[e0 + p]; });
            }
        } else {
            const int m = g.m;
            for (int c = gp.gt; c < m; c += gp.T) {
                const int e0 = EXACT ? c * DC : (int)sg.c_ptr[c];  // check-regular: rows of DC edges
                const int deg = EXACT ? DC : sg.c_ptr[c + 1] - e0;
                const int f = check_node<MASK>(
                    deg, km, kb, writeR, Pc, Pn, [&](int p) { return 4 * (int)sg.c_vn[e0 + p]; },
                    [&](int p) { return (p * m + c) * RSZ; });
                u += f;
            }
        }
        return gp.sum_pass(u);
    }

    __device__ __forceinline__ int vdeg(int v) const {
        if constexpr (QC) return sg.cdeg[v / g.Z];
        else return sg.v_ptr[v + 1] - sg.v_ptr[v];
    }

    // the accumulator: L'(v) = L + beta - dv B in both halves (impulse
    // nodes are patched afterwards)
    // a run of equal words, 16 bytes per store where the run is aligned
    __device__ __forceinline__ void fill(unsigned *row, int count, unsigned w) const {
        if (((uintptr_t)row & 15) == 0 && (count & 3) == 0) {
            uint4 *r4 = (uint4 *)row;
            const uint4 w4 = make_uint4(w, w, w, w);
            for (int k = gp.gt; k < (count >> 2); k += gp.T) r4[k] = w4;
        } else {
            for (int k = gp.gt; k < count; k += gp.T) row[k] = w;
        }
    }
    __device__ __forceinline__ void init_accum(unsigned *Pn, int Lb) const {
        if constexpr (QC) {
            const int Z = g.Z;
            for (int j = 0; j < g.n_b; j++) {
                const unsigned l = (unsigned)(Lb + (int)kBeta - sg.cdeg[j] * pc.B);
                const unsigned l2 = l | (l << 16);
                unsigned *row = Pn + j * Z;
                for (int k = gp.gt; k < Z; k += gp.T) row[k] = l2;
            }
        } else if (g.dv_min == g.dv_max) {  // variable-regular: one value
            const unsigned l = (unsigned)(Lb + (int)kBeta - g.dv_max * pc.B);
            fill(Pn, g.n, l | (l << 16));
        } else {
            for (int v = gp.gt; v < g.n; v += gp.T) {
                const unsigned l = (unsigned)(Lb + (int)kBeta - vdeg(v) * pc.B);
                Pn[v] = l | (l << 16);
            }
        }
    }

    __device__ __forceinline__ static void set_half(unsigned *P, int v, int h, unsigned val) {
        ((uint16_t *)P)[2 * v + h] = (uint16_t)val;
    }
    __device__ __forceinline__ static void add_half(unsigned *P, int v, int h, int delta) {
        uint16_t *q = (uint16_t *)P + 2 * v + h;
        *q = (uint16_t)(*q + delta);
    }

    // the variable-node pass of the VN form (QC): P'(v) = L + beta - dv B +
    // sum of the R' of v's edges in both halves -- the value the accumulating
    // form builds with red.add -- for the baseline channel value L (impulse
    // nodes are corrected afterwards)
    __device__ __forceinline__ void vn_pass(unsigned *P, int Lb) const {
        const int Z = g.Z;
        const unsigned zm = Z > 1 ? 0xFFFFFFFFu / (unsigned)Z + 1u : 0u;  // v / Z = umulhi(v, zm), v < 2^15
        for (int v = gp.gt; v < g.n; v += gp.T) {
            const int j = Z > 1 ? (int)__umulhi((unsigned)v, zm) : v;
            const int k = v - j * Z;
            const int dv = sg.cdeg[j];
            const int32_t *eo = sg.ceoff + j * g.dv_max;
            const int16_t *sh = sg.cs + j * g.dv_max;
            const unsigned l = (unsigned)(Lb + (int)kBeta - dv * pc.B);
            unsigned acc = l | (l << 16);
            for (int t = 0; t < dv; t++) {
                // block (i, j) with shift s joins row r to column (r + s) mod Z: r = (k - s) mod Z
                const int r = wrapZneg(k - sh[t], Z);
                acc += ldR((eo[t] + r) * RSZ);
            }
            P[v] = acc;
        }
    }

    // x_k of half h (P < 0, i.e. bit 15 of the half clear) into a bitmask
    __device__ __forceinline__ void save_x(const unsigned *P, int h, uint32_t *xw) const {
        const unsigned bitpos = 15u + 16u * h;
        for (int base = 0; base < g.n; base += gp.T) {
            const int v = base + gp.gt;
            const bool bit = v < g.n && !((P[v] >> bitpos) & 1u);
            const unsigned w = __ballot_sync(0xffffffffu, bit);
            const int wi = (base >> 5) + gp.gw;
            if (gp.lane == 0 && (wi << 5) < g.n) xw[wi] = w;
        }
    }

    __device__ __forceinline__ int any_neg(const unsigned *P, int h) const {
        const unsigned bitpos = 15u + 16u * h;
        int neg = 0;
        for (int v = gp.gt; v < g.n; v += gp.T) neg |= !((P[v] >> bitpos) & 1u);
        return gp.sum(neg);
    }
};

// The decode loop of one group (G warps, group index grp) over the
// candidate queue of one code; the code's tables are already in sg.
template <bool QC, int DC, bool EXACT, bool I8, bool VN = false>
__device__ void pair_run(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const SlotLayout &lay,
                         int G, const SGraph &sg, unsigned char *smem, int grp) {
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
    unsigned char *Rb = slot + lay.r_off;
    unsigned *Pbuf = (unsigned *)(slot + lay.p_off);  // [2][n] ([n] in the VN form)
    const int nw = (g.n + 31) >> 5;
    uint32_t *xb = (uint32_t *)(slot + lay.xa_off);  // 4 buffers of nw words: [half][cur/keep]
    const int xstride = (nw + 3) & ~3;

    PairConst pc;
    pc.B = I8 ? 128 : 1024;
    pc.sat = dp.sat;
    pc.an = dp.alpha_num;
    pc.as = dp.alpha_shift;
    pc.B2 = (unsigned)pc.B * 0x00010001u;
    pc.BETA2 = kBeta * 0x00010001u;
    pc.BS2 = (kBeta + (unsigned)pc.sat) * 0x00010001u;
    pc.amask2 = (0xFFFFu >> pc.as) * 0x00010001u;
    pc.BAN2 = pc.BETA2 * (unsigned)pc.an;
    // QC codes of check degree 7 or 8 run the all-row-block pass (the row
    // block's shifts read from the tables, not held in registers)
    PairDecoder<QC, DC, EXACT, I8, VN, QC && DC == 8 && !EXACT> dec{g, sg, gp, pc, Rb};

    const long long total = (long long)b.ctr->n_cand_total;
    const long long end = b.cand_end < 0 || b.cand_end > total ? total : b.cand_end;
    const int Lb = clampi(dp.base_llr, -dp.sat, dp.sat);
    const int amax = (1 << dp.amp_steps) - 1;
    long long my_dec = 0, my_it = 0;
    int pcur = 0;  // which posterior buffer holds P_k
    // the converged-decode counts and each half's iteration limit live in the
    // group's shared misc area (written by thread 0 only), not in registers
    if (gp.gt == 0) {
        misc->okd = 0;
        misc->okit = 0;
    }

    Half H[2] = {};  // (every field is set by fetch before use)

    auto fetch = [&](Half &h, int hh) {
        if (gp.gt == 0) misc->bcast[0] = (long long)atomicAdd(b.queue, 1ull);
        gp.sync();
        const long long idx = b.cand_begin + misc->bcast[0];
        gp.sync();
        h.k = 0;
        h.ubest = 0x7fffffff;
        h.first = 1;
        h.cur = 0;
        if (idx >= end) {
            h.idx = -1;
            h.nI = 0;
            return;
        }
        const int4 I4 = b.cands[idx];
        h.idx = idx;
        h.I0 = I4.x; h.I1 = I4.y; h.I2 = I4.z; h.I3 = I4.w;
        h.nI = (I4.x >= 0) + (I4.y >= 0) + (I4.z >= 0) + (I4.w >= 0);
        h.lo = 0; h.hi = amax; h.st = 0; h.phase = 0;
        h.thr = -1; h.ndec = 0; h.nit = 0; h.failed = 0;
        h.Limp = clampi(dp.base_llr - amax, -dp.sat, dp.sat);
        if (gp.gt == 0) misc->K[hh] = cand_limit(dp, b, idx);
        // (read after the next group barrier)
    };
    // finish the candidate of half hh (records, x* to global) and fetch the next
    auto finish = [&](Half &h, int hh) {
        gp.sync();
        const long long o = h.idx - b.rec_base;
        if (h.failed) {
            const uint32_t *src = xb + (2 * hh + (h.cur ^ 1)) * xstride;
            uint32_t *dst = b.xstar + o * (long long)b.nw;
            for (int w = gp.gt; w < nw; w += gp.T) dst[w] = src[w];
        }
        if (gp.gt == 0) {
            b.c_thr[o] = h.failed ? h.thr : -1;
            b.c_thr_f[o] = -1.0f;
            b.c_slot[o] = -1;
            b.c_flags[o] = 0;
            b.c_decodes[o] = h.ndec;
            b.c_iters[o] = h.nit;
        }
        my_dec += h.ndec;
        my_it += h.nit;
        fetch(h, hh);
    };
    // Advance half hh past trivial decodes (impulse LLR >= 0: every hard
    // decision 0, u_0 = 0, success at iteration 0) until a decode that needs
    // iterations is set up (returns true) or no candidate is left.
    auto settle = [&](Half &h, int hh) {
        while (h.idx >= 0) {
            if (h.Limp < 0) return true;
            h.ndec++;
            if (gp.gt == 0) misc->okd++;  // x_0 = 0: converged at iteration 0
            if (h.phase == 0) {
                finish(h, hh);  // no failure at the largest amplitude
                continue;
            }
            h.lo = (h.lo + h.hi) >> 1;  // the decode at mid succeeded
            if (h.st < dp.amp_steps && h.hi - h.lo > 1) {
                const int mid = (h.lo + h.hi) >> 1;
                h.st++;
                h.Limp = clampi(dp.base_llr - mid, -dp.sat, dp.sat);
            } else {
                h.thr = h.hi;
                finish(h, hh);
            }
        }
        return false;
    };
    // half hh of the current posteriors for a new decode: P = L
    auto start_cur = [&](Half &h, int hh, unsigned *Pc) {
        for (int v = gp.gt; v < g.n; v += gp.T) dec.set_half(Pc, v, hh, (unsigned)(Lb + (int)kBeta));
        h.k = 0;
        h.ubest = 0x7fffffff;
        h.first = 1;
    };
    // impulse nodes: the current posteriors (new decode only) and the accumulator
    // the impulse nodes of a new decode in the current posteriors
    auto patch_cur = [&](Half &h, int hh, unsigned *Pc) {
        if (h.idx >= 0 && gp.gt < h.nI) dec.set_half(Pc, h.Ik(gp.gt), hh, (unsigned)(h.Limp + (int)kBeta));
    };
    // The accumulator starts at the baseline L' in every word; its impulse
    // nodes get L_imp - L_base added in their half with the check pass's
    // red.adds (threads 0-3: half 0, 4-7: half 1).  The adds are exact and
    // commute: the word's final halves are in range, so no intermediate
    // carry or borrow between the halves survives.
    auto impulse_adds = [&](unsigned *Pn) {
        if (gp.gt < 8) {  // (the halves selected by value: H stays in registers)
            const int j = gp.gt & 3;
            const bool h1 = gp.gt >= 4;
            const bool on = h1 ? H[1].idx >= 0 && j < H[1].nI : H[0].idx >= 0 && j < H[0].nI;
            const int t = h1 ? H[1].Ik(j) : H[0].Ik(j);
            const unsigned d = (unsigned)((h1 ? H[1].Limp : H[0].Limp) - Lb);
            if (on) red_add((unsigned char *)(Pn + t), h1 ? d << 16 : d);
        }
    };

    // VN form: the impulse nodes of half hh after a variable-node pass (built
    // with the baseline L), or of a new decode
    auto patch_vn = [&](Half &h, int hh, unsigned *Pc, bool fresh) {
        if (h.idx >= 0 && gp.gt < h.nI) {
            const int t = h.Ik(gp.gt);
            if (fresh) dec.set_half(Pc, t, hh, (unsigned)(h.Limp + (int)kBeta));
            else dec.add_half(Pc, t, hh, h.Limp - Lb);
        }
    };

    {
        unsigned *Pc = Pbuf, *Pn = Pbuf + g.n;
        if constexpr (!VN) dec.init_accum(Pn, Lb);
        for (int hh = 0; hh < 2; hh++) {
            fetch(H[hh], hh);
            settle(H[hh], hh);
            start_cur(H[hh], hh, Pc);  // idle halves too: every word stays a valid decode state
        }
        gp.sync();
        for (int hh = 0; hh < 2; hh++) {
            if constexpr (VN) patch_vn(H[hh], hh, Pc, true);
            else patch_cur(H[hh], hh, Pc);
        }
        gp.sync();
    }

    while (H[0].idx >= 0 || H[1].idx >= 0) {
        unsigned *Pc = VN ? Pbuf : Pbuf + pcur * g.n, *Pn = VN ? Pbuf : Pbuf + (pcur ^ 1) * g.n;
        const unsigned km = (H[0].first ? 0xFFFF0000u : 0xFFFFFFFFu) & (H[1].first ? 0x0000FFFFu : 0xFFFFFFFFu);
        const unsigned kb = pc.B2 & ~km;
        const bool wr = (H[0].idx >= 0 && H[0].k < misc->K[0]) || (H[1].idx >= 0 && H[1].k < misc->K[1]);
        // u_k of both halves from P_k = Pc; Pn accumulates P_{k+1}
        if constexpr (!VN) impulse_adds(Pn);
        // (the common form -- no half starting, messages written -- compiled with writeR constant)
        const int us = km != 0xFFFFFFFFu ? dec.template check_pass<true>(km, kb, wr, Pc, Pn)
                       : wr              ? dec.template check_pass<false>(km, kb, true, Pc, Pn)
                                         : dec.template check_pass<false>(km, kb, false, Pc, Pn);
        int restart[2] = {0, 0};
        bool read_pc = false;  // some thread read P_k after the check pass (uniform)
        for (int hh = 0; hh < 2; hh++) {
            Half &h = H[hh];
            if (h.idx < 0) continue;
            const int u = hh == 0 ? (us & 0xFFFF) : (us >> 16);
            uint32_t *xc = xb + (2 * hh + h.cur) * xstride;
            if (h.k >= g.wstart && u < h.ubest) {
                h.ubest = u;
                dec.save_x(Pc, hh, xc);
                read_pc = true;
            }
            if (u != 0 && h.k != misc->K[hh]) continue;
            read_pc = true;
            // the decode ended at K_last = k
            const int kl = h.k;
            if (kl < g.wstart) dec.save_x(Pc, hh, xc);
            const bool fail = u != 0 || dec.any_neg(Pc, hh) != 0;
            h.ndec++;
            h.nit += kl;
            if (!fail && gp.gt == 0) {
                misc->okd++;
                misc->okit += kl;
            }
            if (h.phase == 0) {
                if (!fail) {
                    finish(h, hh);
                } else {
                    h.failed = 1;
                    h.cur ^= 1;
                    h.phase = 1;
                }
            } else {
                const int mid = (h.lo + h.hi) >> 1;
                if (fail) {
                    h.hi = mid;
                    h.cur ^= 1;
                } else {
                    h.lo = mid;
                }
            }
            if (h.idx >= 0 && h.phase == 1) {
                if (h.st < dp.amp_steps && h.hi - h.lo > 1) {
                    const int mid = (h.lo + h.hi) >> 1;
                    h.st++;
                    h.Limp = clampi(dp.base_llr - mid, -dp.sat, dp.sat);
                } else {
                    h.thr = h.hi;
                    finish(h, hh);
                }
            }
            restart[hh] = 1;
        }
        if constexpr (VN) {
            // P_{k+1} from the messages just written, in place of P_k
            gp.sync();
            if (wr) {
                dec.vn_pass(Pc, Lb);
                gp.sync();
            }
            for (int hh = 0; hh < 2; hh++) {
                Half &h = H[hh];
                if (restart[hh]) {
                    if (settle(h, hh)) start_cur(h, hh, Pc);
                } else if (h.idx >= 0) {
                    h.k++;
                    h.first = 0;
                }
            }
            gp.sync();
            for (int hh = 0; hh < 2; hh++) patch_vn(H[hh], hh, Pc, restart[hh] != 0);
            gp.sync();
            continue;
        }
        // Pn (= P_{k+1}) becomes current; the old Pc becomes the next
        // accumulator (a barrier first if P_k was read after the check pass)
        if (read_pc) gp.sync();
        for (int hh = 0; hh < 2; hh++) {
            Half &h = H[hh];
            if (restart[hh]) {
                if (settle(h, hh)) start_cur(h, hh, Pn);
            } else if (h.idx >= 0) {
                h.k++;
                h.first = 0;
            }
        }
        dec.init_accum(Pc, Lb);
        if (restart[0] | restart[1]) {
            gp.sync();  // after start_cur's stores
            for (int hh = 0; hh < 2; hh++)
                if (restart[hh]) patch_cur(H[hh], hh, Pn);
        }
        gp.sync();
        pcur ^= 1;
    }
    if (gp.gt == 0) {
        atomicAdd(&b.ctr->decodes, (unsigned long long)my_dec);
        atomicAdd(&b.ctr->iterations, (unsigned long long)my_it);
        atomicAdd(&b.ctr->edge_updates, (unsigned long long)my_it * (unsigned long long)g.E);
        atomicAdd(&b.ctr->ok_decodes, misc->okd);
        atomicAdd(&b.ctr->ok_iters, misc->okit);
    }
}

template <bool QC, int DC, bool EXACT, bool I8>
__global__ void __launch_bounds__(32 * pair_kernel_warps(QC, DC, EXACT))
    pair_kernel(DevCode g, DecodeParams dp, EnumBuffers b, SlotLayout lay, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem, true);
    __syncthreads();
    pair_run<QC, DC, EXACT, I8>(g, dp, b, lay, G, sg, smem, (threadIdx.x >> 5) / G);
}

// the VN form for QC codes of large check degree whose two-buffer layout does not fit
template <bool I8>
__global__ void __launch_bounds__(32 * kPairWarps) pair_vn_kernel(DevCode g, DecodeParams dp, EnumBuffers b,
                                                               SlotLayout lay, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SGraph sg = load_tables(g, smem, true);
    __syncthreads();
    pair_run<true, 32, false, I8, true>(g, dp, b, lay, G, sg, smem, (threadIdx.x >> 5) / G);
}

// One persistent launch over several codes: every CTA works through the
// codes in order, each with its own tables, slot layout and group size,
// taking candidates from that code's queue until it is empty (CTAs move
// on independently, so no code waits for the slowest CTA of another).
// The items are a __grid_constant__ kernel parameter: the decoders read
// each code's description from the constant bank, as the single-code kernel
// does, instead of holding it in registers.
template <bool QC, int DC, bool EXACT, bool I8>
__global__ void __launch_bounds__(512) batch_kernel(const __grid_constant__ BatchArgs args, int n_items) {
    extern __shared__ __align__(16) unsigned char smem[];
    for (int c = 0; c < n_items; c++) {
        const BatchItem &it = args.it[c];
        const SGraph sg = load_tables(it.g, smem, true);
        __syncthreads();
        const int grp = (threadIdx.x >> 5) / it.G;
        if (grp < it.groups) pair_run<QC, DC, EXACT, I8>(it.g, it.dp, it.b, it.lay, it.G, sg, smem, grp);
        __syncthreads();
    }
}

template <bool I8>
cudaError_t launch_pair(const DevCode &g, const DecodeParams &dp, const EnumBuffers &b, const LaunchShape &sh,
                        cudaStream_t st) {
    const bool qc = g.kind == TSX_CODE_QC;
    const bool reg6 = g.dc_min == 6 && g.dc_max == 6;
    if (reg6)
        return qc ? launch_persistent(pair_kernel<true, 6, true, I8>, sh, st, g, dp, b, sh.lay, sh.G)
                  : launch_persistent(pair_kernel<false, 6, true, I8>, sh, st, g, dp, b, sh.lay, sh.G);
    if (g.dc_max <= 8)
        return qc ? launch_persistent(pair_kernel<true, 8, false, I8>, sh, st, g, dp, b, sh.lay, sh.G)
                  : launch_persistent(pair_kernel<false, 8, false, I8>, sh, st, g, dp, b, sh.lay, sh.G);
    return qc ? launch_persistent(pair_kernel<true, 32, false, I8>, sh, st, g, dp, b, sh.lay, sh.G)
              : launch_persistent(pair_kernel<false, 32, false, I8>, sh, st, g, dp, b, sh.lay, sh.G);
}

template <bool I8>
cudaError_t launch_batch_t(const BatchArgs &items, int n, bool qc, int dc_max, bool reg6, const LaunchShape &sh,
                           cudaStream_t st) {
    if (reg6)
        return qc ? launch_persistent(batch_kernel<true, 6, true, I8>, sh, st, items, n)
                  : launch_persistent(batch_kernel<false, 6, true, I8>, sh, st, items, n);
    if (dc_max <= 8)
        return qc ? launch_persistent(batch_kernel<true, 8, false, I8>, sh, st, items, n)
                  : launch_persistent(batch_kernel<false, 8, false, I8>, sh, st, items, n);
    return qc ? launch_persistent(batch_kernel<true, 32, false, I8>, sh, st, items, n)
              : launch_persistent(batch_kernel<false, 32, false, I8>, sh, st, items, n);
}

}  // namespace
}  // namespace tsx
