// cycles.cu -- short cycles of the Tanner graph on the device: the EMD
// spectrum of Sec. II (Table II) and the per-node cycle counts behind the
// cycle-density iteration budgets of Sec. III (Table V).
//
// A cycle of length 2l is an exponent chain that closes (Prop. 1, eq. 3): a
// closed walk v0 - c1 - v1 - ... - v_{l-1} - c_l - v0 that never steps
// straight back (c_{t+1} != c_t, v_{t+1} != v_t, c_l != c_1), up to rotation
// and reversal; it may pass a node twice.  Walked from a representative v0
// ((j,0) of a QC code, every node of a general code), the column index of
// every node of a QC walk is the running alternating sum of the exponents,
// and the walk closes exactly when that sum is 0 mod Z.  A walk class with
// rotation period p and r = 1 (its reverse is a rotation) or 2 is met p r
// times over the representatives (per circulant orbit, for a QC code); each
// walk adds 2l / (p r) to hist2[l][EMD], so hist2 / (2l) counts classes --
// Table II's "number of cycles without multiplication by graph automorphism".
// For l <= 3 every such walk is a simple cycle: walks from v of length 2l
// are twice the cycles through v.
//
// The EMD is the number of checks meeting exactly one variable node of the
// walk.  One thread walks every continuation of one two-step prefix
// (v0, c1, v1, c2, v2) with an explicit stack; lengths up to 2 kLmax.
#include "graph.cuh"
#include "kernels.cuh"

namespace tsx {
namespace {

constexpr int kLmax = kCycLmax;

__device__ __forceinline__ bool has_check(const DevCode &g, int v, int c) {
    const int d = vn_degree(g, v);
    for (int t = 0; t < d; t++)
        if (vn_check(g, v, t) == c) return true;
    return false;
}

// checks meeting exactly one distinct variable node of vs[0..L-1]
__device__ int emd_of(const DevCode &g, const int *vs, int L) {
    int u[kLmax], nu = 0;
    for (int x = 0; x < L; x++) {
        bool dup = false;
        for (int y = 0; y < nu; y++) dup |= u[y] == vs[x];
        if (!dup) u[nu++] = vs[x];
    }
    int emd = 0;
    for (int x = 0; x < nu; x++) {
        const int d = vn_degree(g, u[x]);
        for (int t = 0; t < d; t++) {
            const int c = vn_check(g, u[x], t);
            bool other = false;
            for (int y = 0; y < nu && !other; y++)
                if (y != x) other = has_check(g, u[y], c);
            emd += !other;
        }
    }
    return emd;
}

// p r of the closed walk vs[0..L-1], cs[1..L] (cs[t] joins vs[t-1] and vs[t mod L])
__device__ int walk_reps(const int *vs, const int *cs, int L) {
    int p = L;
    for (int q = 1; q < L; q++) {
        if (L % q) continue;
        bool ok = true;
        for (int t = 0; t < L && ok; t++) ok = vs[(t + q) % L] == vs[t] && cs[(t + q) % L + 1] == cs[t + 1];
        if (ok) {
            p = q;
            break;
        }
    }
    // the reverse rotated by s: v_{(s-t) mod L} followed by c_{(s-t) mod L} (c_0 = c_L)
    int r = 2;
    for (int sft = 0; sft < L && r == 2; sft++) {
        bool ok = true;
        for (int t = 0; t < L && ok; t++) {
            const int a = ((sft - t) % L + L) % L;
            ok = vs[a] == vs[t] && cs[a == 0 ? L : a] == cs[t + 1];
        }
        if (ok) r = 1;
    }
    return p * r;
}

// walks[rep * (kLmax + 1) + l]: closed walks of l variable nodes from the
// representative; hist2[l * kEmdBins + e]: sum of 2l / (p r) over them by EMD.
// Thread id = (rep, t_1, p_1, ..., t_pd, p_pd): the walk's first pd steps
// (check t of the last node, then node p of that check); the walks that
// close within the prefix are counted by the thread whose deeper indices are
// all 0, and the rest of the search runs from the prefix's last node.
__global__ void __launch_bounds__(256) cycle_kernel(DevCode g, int lmax, int pd, long long n_prefix,
                                                    unsigned long long *walks, unsigned long long *hist2) {
    const int dvm = g.dv_max, dcm = g.dc_max;
    for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n_prefix;
         id += (long long)gridDim.x * blockDim.x) {
        long long x = id;
        int tt[4], pp[4];
        for (int lvl = pd; lvl >= 1; lvl--) {
            pp[lvl] = (int)(x % dcm);
            x /= dcm;
            tt[lvl] = (int)(x % dvm);
            x /= dvm;
        }
        const int rep = (int)x;
        int vs[kLmax], cs[kLmax + 1];
        vs[0] = rep_vn(g, rep);
        unsigned long long cnt[kLmax + 1] = {0, 0, 0, 0, 0, 0, 0};
        // the walks that close at v_d through a check of v_d holding v0
        auto closure = [&](int d) {
            if (vs[d] == vs[0]) return;
            const int dv = vn_degree(g, vs[d]);
            for (int t = 0; t < dv; t++) {
                const int c = vn_check(g, vs[d], t);
                if (c == cs[d] || c == cs[1] || !has_check(g, vs[0], c)) continue;
                const int L = d + 1;
                cs[L] = c;
                cnt[L]++;
                if (hist2) atomicAdd(&hist2[L * kEmdBins + emd_of(g, vs, L)], (unsigned long long)(2 * L / walk_reps(vs, cs, L)));
            }
        };
        int d = 0;
        bool ok = true;
        for (int lvl = 1; lvl <= pd && ok; lvl++) {
            const int v = vs[lvl - 1];
            if (tt[lvl] >= vn_degree(g, v)) { ok = false; break; }
            const int c = vn_check(g, v, tt[lvl]);
            if (lvl > 1 && c == cs[lvl - 1]) { ok = false; break; }
            if (pp[lvl] >= cn_degree(g, c)) { ok = false; break; }
            const int u = cn_vn(g, c, pp[lvl]);
            if (u == v) { ok = false; break; }
            cs[lvl] = c;
            vs[lvl] = u;
            d = lvl;
            bool zero_below = true;
            for (int l2 = lvl + 1; l2 <= pd; l2++) zero_below = zero_below && tt[l2] == 0 && pp[l2] == 0;
            if (zero_below) closure(lvl);
            if (lvl >= lmax - 1) {  // no longer walk needed; deeper prefix indices count nothing
                ok = zero_below;
                break;
            }
        }
        if (ok && d == pd && d < lmax - 1) {
            int ti[kLmax], pi[kLmax];
            ti[d] = 0;
            pi[d] = 0;
            bool enter = false;  // the prefix's last node is counted already
            while (d >= pd) {
                if (enter) {
                    closure(d);
                    if (d >= lmax - 1) {
                        d--;
                        enter = false;
                        continue;
                    }
                    ti[d] = 0;
                    pi[d] = 0;
                }
                bool pushed = false;
                const int dv = vn_degree(g, vs[d]);
                while (ti[d] < dv && !pushed) {
                    const int c = vn_check(g, vs[d], ti[d]);
                    if (c != cs[d]) {
                        const int dc = cn_degree(g, c);
                        while (pi[d] < dc) {
                            const int u = cn_vn(g, c, pi[d]);
                            pi[d]++;
                            if (u != vs[d]) {
                                cs[d + 1] = c;
                                vs[d + 1] = u;
                                pushed = true;
                                break;
                            }
                        }
                    }
                    if (!pushed) {
                        ti[d]++;
                        pi[d] = 0;
                    }
                }
                if (pushed) {
                    d++;
                    enter = true;
                } else {
                    d--;
                    enter = false;
                }
            }
        }
        for (int L = 2; L <= lmax; L++)
            if (cnt[L]) atomicAdd(&walks[rep * (kLmax + 1) + L], cnt[L]);
    }
}

}  // namespace

// Closed walks per representative and length (walks[n_rep][kLmax + 1]) and,
// if hist is not null, the class-weighted counts per length and EMD
// (hist[kLmax + 1][kEmdBins]); both zeroed here.
cudaError_t launch_cycles(const DevCode &g, int lmax, unsigned long long *walks, unsigned long long *hist,
                          cudaStream_t st) {
    if (lmax < 2 || lmax > kLmax) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(walks, 0, sizeof(unsigned long long) * g.n_rep * (kLmax + 1), st);
    if (e != cudaSuccess) return e;
    if (hist && (e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * (kLmax + 1) * kEmdBins, st)) !=
                    cudaSuccess)
        return e;
    // three-step prefixes for the deep searches (more, shorter subtrees), two otherwise
    const int pd = lmax >= 5 ? 3 : 2;
    long long n_prefix = g.n_rep;
    for (int l = 0; l < pd; l++) n_prefix *= (long long)g.dv_max * g.dc_max;
    long long blocks = (n_prefix + 255) / 256;
    if (blocks > 1 << 20) blocks = 1 << 20;
    cycle_kernel<<<(int)blocks, 256, 0, st>>>(g, lmax, pd, n_prefix, walks, hist);
    return cudaGetLastError();
}

}  // namespace tsx
