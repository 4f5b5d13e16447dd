// cand.cu -- Tanner balls and candidate impulse sets, on the device.
//
// Sec. III: for every orbit representative VN1 a depth-3 tree
// VN1-CN1-VN2-CN2-VN3 is unrolled and impulse sets are drawn from its
// variable layers.  The library's candidate rule: sets {rep} u T with T a
// subset of the representative's Tanner ball (variable nodes at distance 2
// or 4), |T| <= max_size - 1, plus (cycle_len = 2l > 2 max_size) the
// variable-node sets of the 2l-cycles through the representative.  One set
// per circulant-shift orbit is decoded (Sec. III, "graph automorphism").
//
// Exactly-once emission without a hash table: a raw set is the pair (rep,
// S).  The raw pairs of one orbit are (rep(y), S shifted so that y has
// k = 0) for every member y whose Tanner ball holds all other members.  A raw
// pair is emitted only if it is the smallest of its orbit's raw pairs in
// the order (sorted tuple, block of y) -- for general codes: only from its
// smallest qualifying member.  The emitted record is the set's canonical
// key (the smallest sorted tuple over the shifts that move a member to
// k = 0), so the output equals the sorted-unique list of canonical keys, in
// a deterministic order (representative, then raw index).
#include "graph.cuh"
#include "kernels.cuh"

namespace tsx {

// ------------------------------------------------------------------------
// Tanner balls
// ------------------------------------------------------------------------
template <bool WRITE>
__global__ void __launch_bounds__(256) ball_kernel(DevCode g, int *sizes, const int64_t *ptr,
                                                   int32_t *ball) {
    extern __shared__ uint32_t bits[];  // [nw] + level-2 list
    const int nw = (g.n + 31) >> 5;
    int *lvl2 = (int *)(bits + nw);
    __shared__ int n2;
    const int rep = blockIdx.x;
    const int v0 = rep_vn(g, rep);
    for (int w = threadIdx.x; w < nw; w += blockDim.x) bits[w] = 0;
    if (threadIdx.x == 0) n2 = 0;
    __syncthreads();
    const int dv0 = vn_degree(g, v0);
    if (threadIdx.x == 0) {
        for (int t = 0; t < dv0; t++) {
            int c = vn_check(g, v0, t);
            int dc = cn_degree(g, c);
            for (int p = 0; p < dc; p++) {
                int u = cn_vn(g, c, p);
                if (u == v0) continue;
                unsigned m = 1u << (u & 31);
                if (!(bits[u >> 5] & m)) {
                    bits[u >> 5] |= m;
                    lvl2[n2++] = u;
                }
            }
        }
    }
    __syncthreads();
    // level 4: everything adjacent to level 2 (parallel over level-2 nodes)
    for (int idx = threadIdx.x; idx < n2; idx += blockDim.x) {
        int u = lvl2[idx];
        int du = vn_degree(g, u);
        for (int t = 0; t < du; t++) {
            int c = vn_check(g, u, t);
            int dc = cn_degree(g, c);
            for (int p = 0; p < dc; p++) {
                int w = cn_vn(g, c, p);
                if (w != v0) atomicOr(&bits[w >> 5], 1u << (w & 31));
            }
        }
    }
    __syncthreads();
    if (!WRITE) {
        int cnt = 0;
        for (int w = threadIdx.x; w < nw; w += blockDim.x) cnt += __popc(bits[w]);
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        __shared__ int tot;
        if (threadIdx.x == 0) tot = 0;
        __syncthreads();
        if ((threadIdx.x & 31) == 0) atomicAdd(&tot, cnt);
        __syncthreads();
        if (threadIdx.x == 0) sizes[rep] = tot;
        return;
    }
    // ordered compaction: one thread walks the words (balls are small)
    if (threadIdx.x == 0) {
        int64_t o = ptr[rep];
        for (int w = 0; w < nw; w++) {
            uint32_t x = bits[w];
            while (x) {
                int b = __ffs(x) - 1;
                x &= x - 1;
                ball[o++] = w * 32 + b;
            }
        }
    }
}

int ball_smem_bytes(const DevCode &g) {
    int nw = (g.n + 31) / 32;
    return nw * 4 + g.dv_max * g.dc_max * 4 + 16;
}

cudaError_t launch_ball(const DevCode &g, int *sizes, const int64_t *ptr, int32_t *ball, bool write,
                        cudaStream_t st) {
    int smem = ball_smem_bytes(g);
    if (write)
        ball_kernel<true><<<g.n_rep, 256, smem, st>>>(g, sizes, ptr, ball);
    else
        ball_kernel<false><<<g.n_rep, 256, smem, st>>>(g, sizes, ptr, ball);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------
// raw set decoding and the emission rule
// ------------------------------------------------------------------------
__device__ __forceinline__ long long choose2(long long n) { return n * (n - 1) / 2; }
__device__ __forceinline__ long long choose3(long long n) { return n * (n - 1) * (n - 2) / 6; }

// pairs (i<j) of [0,nb) in lexicographic order: index q -> (i, j)
__device__ void unrank2(long long q, int nb, int &i, int &j) {
    long long tot = choose2(nb);
    int lo = 0, hi = nb - 2;  // largest i with (tot - C(nb-i,2)) <= q
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tot - choose2(nb - mid) <= q) lo = mid;
        else hi = mid - 1;
    }
    i = lo;
    j = i + 1 + (int)(q - (tot - choose2(nb - i)));
}
__device__ void unrank3(long long q, int nb, int &i, int &j, int &k) {
    long long tot = choose3(nb);
    int lo = 0, hi = nb - 3;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (tot - choose3(nb - mid) <= q) lo = mid;
        else hi = mid - 1;
    }
    i = lo;
    long long r = q - (tot - choose3(nb - i));
    int a, b;
    unrank2(r, nb - i - 1, a, b);
    j = i + 1 + a;
    k = i + 1 + b;
}

__device__ __forceinline__ void sort_small(int *x, int n) {
    for (int a = 1; a < n; a++) {
        int v = x[a], b = a - 1;
        while (b >= 0 && x[b] > v) { x[b + 1] = x[b]; b--; }
        x[b + 1] = v;
    }
}
__device__ __forceinline__ int lex_cmp(const int *a, const int *b, int n) {
    for (int i = 0; i < n; i++)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}

__device__ bool in_ball(const DevCode &g, int rep, int v) {
    int64_t lo = g.ball_ptr[rep], hi = g.ball_ptr[rep + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        int x = g.ball[mid];
        if (x == v) return true;
        if (x < v) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

// is t in the Tanner ball of y?
__device__ bool near_vn(const DevCode &g, int y, int t) {
    if (g.kind == TSX_CODE_QC) {
        int jy = y / g.Z, ky = y - jy * g.Z;
        return in_ball(g, jy, shift_vn(g, t, -ky));
    }
    return in_ball(g, y, t);
}

// canonical key of a set of <= 4 nodes: smallest sorted tuple among the
// shifts moving a member to k = 0 (sorted set for general codes)
__device__ void canon_small(const DevCode &g, const int *S, int n, int *key) {
    for (int i = 0; i < n; i++) key[i] = S[i];
    sort_small(key, n);
    if (g.kind != TSX_CODE_QC) return;
    int tmp[4];
    bool have = false;
    for (int y = 0; y < n; y++) {
        int ky = S[y] % g.Z;
        for (int i = 0; i < n; i++) tmp[i] = shift_vn(g, S[i], -ky);
        sort_small(tmp, n);
        if (!have || lex_cmp(tmp, key, n) < 0) {
            for (int i = 0; i < n; i++) key[i] = tmp[i];
            have = true;
        }
    }
}

// Emission rule for the raw pair (rep, S), S[0] = rep node, |S| = n.
__device__ bool emit_rule(const DevCode &g, int rep, const int *S, int n) {
    if (n == 1) return true;
    if (g.kind == TSX_CODE_QC) {
        int ours[4], tmp[4];
        for (int i = 0; i < n; i++) ours[i] = S[i];
        sort_small(ours, n);
        const int jr = rep;
        for (int y = 1; y < n; y++) {
            bool q = true;  // S[0] is in y's ball (y is in rep's ball)
            for (int t = 1; t < n && q; t++)
                if (t != y) q = near_vn(g, S[y], S[t]);
            if (!q) continue;
            int jy = S[y] / g.Z, ky = S[y] - jy * g.Z;
            for (int i = 0; i < n; i++) tmp[i] = shift_vn(g, S[i], -ky);
            sort_small(tmp, n);
            int c = lex_cmp(tmp, ours, n);
            if (c < 0 || (c == 0 && jy < jr)) return false;
        }
        return true;
    }
    for (int y = 1; y < n; y++) {
        if (S[y] > S[0]) continue;
        bool q = true;
        for (int t = 1; t < n && q; t++)
            if (t != y) q = near_vn(g, S[y], S[t]);
        if (q) return false;
    }
    return true;
}

// raw local index q of representative rep -> set S (S[0] = rep node)
__device__ int raw_set(const DevCode &g, int rep, long long q, int *S) {
    const int64_t b0 = g.ball_ptr[rep];
    const int nb = (int)(g.ball_ptr[rep + 1] - b0);
    S[0] = rep_vn(g, rep);
    if (q == 0) return 1;
    q -= 1;
    if (q < nb) {
        S[1] = g.ball[b0 + q];
        return 2;
    }
    q -= nb;
    long long c2 = choose2(nb);
    if (q < c2) {
        int i, j;
        unrank2(q, nb, i, j);
        S[1] = g.ball[b0 + i];
        S[2] = g.ball[b0 + j];
        return 3;
    }
    q -= c2;
    int i, j, k;
    unrank3(q, nb, i, j, k);
    S[1] = g.ball[b0 + i];
    S[2] = g.ball[b0 + j];
    S[3] = g.ball[b0 + k];
    return 4;
}

constexpr int kChunk = 1024;  // raw sets per CTA
constexpr int kCandThreads = 256;

template <bool WRITE>
__global__ void __launch_bounds__(kCandThreads) cand_ball_kernel(CandArgs a) {
    const long long base = (long long)blockIdx.x * kChunk;
    const int per = kChunk / kCandThreads;
    int keys[4][4];
    int sizes[4];
    int cnt = 0;
    for (int u = 0; u < per; u++) {
        long long raw = base + (long long)threadIdx.x * per + u;
        sizes[u] = 0;
        if (raw >= a.raw_total) continue;
        int lo = 0, hi = a.code.n_rep - 1;  // rep with raw_off[rep] <= raw
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (a.raw_off[mid] <= raw) lo = mid;
            else hi = mid - 1;
        }
        int S[4];
        int n = raw_set(a.code, lo, raw - a.raw_off[lo], S);
        if (!emit_rule(a.code, lo, S, n)) continue;
        sizes[u] = n;
        if (WRITE) canon_small(a.code, S, n, keys[u]);
        cnt++;
    }
    // block-wide exclusive scan of cnt (thread order = raw order)
    __shared__ int warp_tot[kCandThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int woff = 0, tot = 0;
    for (int w = 0; w < kCandThreads / 32; w++) {
        if (w < wid) woff += warp_tot[w];
        tot += warp_tot[w];
    }
    if (!WRITE) {
        if (threadIdx.x == 0) a.chunk_count[blockIdx.x] = tot;
        return;
    }
    long long pos = a.chunk_off[blockIdx.x] + woff + incl - cnt;
    for (int u = 0; u < per; u++) {
        if (!sizes[u]) continue;
        int n = sizes[u];
        int4 r = make_int4(keys[u][0], n > 1 ? keys[u][1] : -1, n > 2 ? keys[u][2] : -1,
                           n > 3 ? keys[u][3] : -1);
        a.cands[pos++] = r;
    }
}

// Exclusive scan of chunk counts (single CTA), appends the grand total.
__global__ void __launch_bounds__(1024) scan_kernel(const int *cnt, long long n, long long *off,
                                                    const long long *base, Counters *ctr, int add_total) {
    __shared__ long long part[32];
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = base ? *base : 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long s = 0; s < n; s += blockDim.x) {
        long long i = s + threadIdx.x;
        long long x = i < n ? cnt[i] : 0;
        long long incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) part[wid] = incl;
        __syncthreads();
        long long woff = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) {
            if (w < wid) woff += part[w];
            tot += part[w];
        }
        if (i < n) off[i] = carry + woff + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[n] = carry;
        if (add_total) ctr->n_cand_total = (unsigned long long)carry;
    }
}

cudaError_t launch_cand_ball(const CandArgs &a, long long n_chunks, bool write, cudaStream_t st) {
    if (n_chunks <= 0) return cudaSuccess;
    if (write)
        cand_ball_kernel<true><<<(unsigned)n_chunks, kCandThreads, 0, st>>>(a);
    else
        cand_ball_kernel<false><<<(unsigned)n_chunks, kCandThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const int *cnt, long long n, long long *off, const long long *base, Counters *ctr,
                        bool add_total, cudaStream_t st) {
    scan_kernel<<<1, 1024, 0, st>>>(cnt, n, off, base, ctr, add_total ? 1 : 0);
    return cudaGetLastError();
}

long long cand_chunks(long long raw_total) { return (raw_total + kChunk - 1) / kChunk; }

// ------------------------------------------------------------------------
// cycle sets: the variable nodes of the 2l-cycles through a representative
// ------------------------------------------------------------------------
constexpr int kCycCap = 2048;
constexpr int kCycThreads = 256;

// path index -> cycle; returns the number of VNs (l) if the path closes
// into a simple 2l-cycle through v0, else 0.
__device__ int cycle_from_index(const DevCode &g, int v0, int l, long long idx, int *vs) {
    int cs[4];
    vs[0] = v0;
    int v = v0, cin = -1;
    for (int step = 0; step < l; step++) {
        int dvv = vn_degree(g, v);
        int tsel = (int)(idx % g.dv_max);
        idx /= g.dv_max;
        if (tsel >= dvv) return 0;
        int c = vn_check(g, v, tsel);
        if (c == cin) return 0;
        for (int s = 0; s < step; s++)
            if (cs[s] == c) return 0;
        cs[step] = c;
        if (step == l - 1) {
            // the last check must close the cycle at v0: c adjacent to v0
            int d0 = vn_degree(g, v0);
            bool ok = false;
            for (int t = 0; t < d0; t++) ok |= vn_check(g, v0, t) == c;
            return ok ? l : 0;
        }
        int dcc = cn_degree(g, c);
        int psel = (int)(idx % g.dc_max);
        idx /= g.dc_max;
        if (psel >= dcc) return 0;
        int u = cn_vn(g, c, psel);
        if (u == v) return 0;
        for (int s = 0; s <= step; s++)
            if (vs[s] == u) return 0;
        vs[step + 1] = u;
        v = u;
        cin = c;
    }
    return 0;
}

__device__ __forceinline__ bool key_less(const int4 &a, const int4 &b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    if (a.z != b.z) return a.z < b.z;
    return a.w < b.w;
}

// One CTA per representative.  WRITE=false: count distinct emitted sets;
// WRITE=true: write them sorted at off[rep].
template <bool WRITE>
__global__ void __launch_bounds__(kCycThreads) cand_cycle_kernel(CycleArgs a) {
    __shared__ int4 list[kCycCap];
    __shared__ int nlist;
    const int rep = blockIdx.x;
    const DevCode &g = a.code;
    const int v0 = rep_vn(g, rep);
    if (threadIdx.x == 0) nlist = 0;
    __syncthreads();
    for (long long idx = threadIdx.x; idx < a.paths; idx += blockDim.x) {
        int vs[4];
        int l = cycle_from_index(g, v0, a.l, idx, vs);
        if (!l) continue;
        // rep(y) for every member y; every member lies on the cycle, so all qualify
        int ours[4], tmp[4];
        for (int i = 0; i < l; i++) ours[i] = vs[i];
        sort_small(ours, l);
        bool emit = true;
        if (g.kind == TSX_CODE_QC) {
            for (int y = 1; y < l && emit; y++) {
                int jy = vs[y] / g.Z, ky = vs[y] - jy * g.Z;
                for (int i = 0; i < l; i++) tmp[i] = shift_vn(g, vs[i], -ky);
                sort_small(tmp, l);
                int c = lex_cmp(tmp, ours, l);
                if (c < 0 || (c == 0 && jy < rep)) emit = false;
            }
        } else {
            for (int y = 1; y < l; y++) emit &= vs[y] > v0;
        }
        if (!emit) continue;
        int key[4];
        canon_small(g, vs, l, key);
        int4 k4 = make_int4(key[0], l > 1 ? key[1] : -1, l > 2 ? key[2] : -1, l > 3 ? key[3] : -1);
        int slot = atomicAdd(&nlist, 1);
        if (slot < kCycCap) list[slot] = k4;
        else atomicOr(&a.ctr->err, kErrCycleOverflow);
    }
    __syncthreads();
    int nl = min(nlist, kCycCap);
    // keep the first copy of equal entries, then place each kept entry at
    // its rank among the kept ones (sorted, deterministic output)
    __shared__ unsigned char keep[kCycCap];
    __shared__ int nuniq;
    if (threadIdx.x == 0) nuniq = 0;
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
        int4 x = list[i];
        bool first = true;
        for (int j = 0; j < i && first; j++) {
            int4 y = list[j];
            if (y.x == x.x && y.y == x.y && y.z == x.z && y.w == x.w) first = false;
        }
        keep[i] = first;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
        if (!keep[i]) continue;
        atomicAdd(&nuniq, 1);
        if (WRITE) {
            int4 x = list[i];
            int rank = 0;
            for (int j = 0; j < nl; j++) rank += keep[j] && key_less(list[j], x);
            a.cands[a.off[rep] + rank] = x;
        }
    }
    __syncthreads();
    if (!WRITE && threadIdx.x == 0) a.count[rep] = nuniq;
}

cudaError_t launch_cand_cycle(const CycleArgs &a, bool write, cudaStream_t st) {
    if (write)
        cand_cycle_kernel<true><<<a.code.n_rep, kCycThreads, 0, st>>>(a);
    else
        cand_cycle_kernel<false><<<a.code.n_rep, kCycThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tsx

namespace tsx {

// ------------------------------------------------------------------------
// cycle-density iteration budgets (Sec. III: fewer iterations where short
// cycles are dense): K(I) = kmin + ceil((K - kmin) wref / (wref + W(I))),
// W(I) = sum over v in I of vweight[v] = 2 c4(v) + c6(v)
// ------------------------------------------------------------------------
__global__ void budget_kernel(const int4 *cands, long long bound, const int *vweight, int K, int kmin, int wref,
                              uint16_t *cand_K, const Counters *ctr) {
    const long long total = (long long)ctr->n_cand_total;
    const long long n = total < bound ? total : bound;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int4 c = cands[i];
        long long W = 0;
        if (c.x >= 0) W += vweight[c.x];
        if (c.y >= 0) W += vweight[c.y];
        if (c.z >= 0) W += vweight[c.z];
        if (c.w >= 0) W += vweight[c.w];
        const long long den = (long long)wref + W;
        cand_K[i] = (uint16_t)(kmin + (((long long)(K - kmin) * wref + den - 1) / den));
    }
}

cudaError_t launch_budget(const int4 *cands, long long bound, const int *vweight, int K, int kmin, int wref,
                          uint16_t *cand_K, const Counters *ctr, cudaStream_t st) {
    long long blocks = (bound + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    budget_kernel<<<(int)blocks, 256, 0, st>>>(cands, bound, vweight, K, kmin, wref, cand_K, ctr);
    return cudaGetLastError();
}

}  // namespace tsx
