/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the modified Cole
 * impulse method of Usatyuk, "An Modified Cole's Importance Sampling Method
 * For Low Error Floor QC-LDPC Codes Construction" (arXiv 2208.05795), used
 * to check the CUDA library.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg may load it; the library never does, and this
 * file shares no code, header or table with the library.
 *
 * Every function states the passage it follows.  Where the paper leaves a
 * choice open the reading taken is stated beside the code.
 *
 * Parity status:
 *   graph expansion (eqs. 1-2)          pinned (Table II / Table V counts)
 *   girth, Tanner ball                  pinned (BFS on hand-drawn graphs, Table III caption)
 *   Tree()/TS(), (a,b), orbit           pinned (Table III TS(2,2)=TS(3,2)=128 by brute force)
 *   canonical key                       pinned (brute force over all shifts)
 *   min-sum decoder                     hand-computed iteration trace; codeword fixed point
 *   sum-product decoder                 exact MAP on a cycle-free code
 *   bisection                           linear scan on the tiny code
 *   importance-sampling weights         closed forms (mu = 0, Gaussian moments)
 *   best pattern x*                     first minimum in the window, on recounted u_k traces
 *   IS channel quantizer                ties / saturation; LLRs recomputed from the normals
 *   ordered list over iterations        dense-matrix restatement on the decoder's x_k trace;
 *                                       two-stage kstart from recounted converged decodes
 *   layered simulation decoder          hand-computed iterations; QC layer = its rows one by one;
 *                                       saturation of each width; codeword inputs; frame channel
 *   cycles, EMD (Prop. 1)               Table II rows 4-10 (Code 1); Hashimoto-matrix traces;
 *                                       brute-force walk classes; Table V densities
 *   iteration budgets                   per-candidate rerun with K = K(I)
 * The decoders themselves are not specified by the paper ("our used version
 * of message passing decoder", Sec. III), so the decoder arithmetic has no
 * paper pin beyond the substitutes above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Tanner graph                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    int n, m, E;
    int Z;          /* circulant size; 0 for a general (non-QC) code */
    int n_b, m_b;
    int dvmax, dcmax;
    int *vdeg, *vadj, *vpos; /* checks of v ascending; vpos = position of v in that check */
    int *cdeg, *cadj;        /* variable nodes of c ascending */
    int girth;               /* 0 until computed */
} og_graph;

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

static og_graph *graph_from_edges(int n, int m, int E, const int *ec, const int *ev) {
    og_graph *g = (og_graph *)calloc(1, sizeof(og_graph));
    g->n = n; g->m = m; g->E = E;
    g->vdeg = (int *)calloc(n, sizeof(int));
    g->cdeg = (int *)calloc(m, sizeof(int));
    for (int e = 0; e < E; e++) { g->vdeg[ev[e]]++; g->cdeg[ec[e]]++; }
    g->dvmax = 1; g->dcmax = 1;
    for (int v = 0; v < n; v++) if (g->vdeg[v] > g->dvmax) g->dvmax = g->vdeg[v];
    for (int c = 0; c < m; c++) if (g->cdeg[c] > g->dcmax) g->dcmax = g->cdeg[c];
    g->vadj = (int *)malloc(sizeof(int) * (size_t)n * g->dvmax);
    g->vpos = (int *)malloc(sizeof(int) * (size_t)n * g->dvmax);
    g->cadj = (int *)malloc(sizeof(int) * (size_t)m * g->dcmax);
    int *fv = (int *)calloc(n, sizeof(int)), *fc = (int *)calloc(m, sizeof(int));
    for (int e = 0; e < E; e++) {
        g->vadj[ev[e] * g->dvmax + fv[ev[e]]++] = ec[e];
        g->cadj[ec[e] * g->dcmax + fc[ec[e]]++] = ev[e];
    }
    for (int v = 0; v < n; v++) qsort(g->vadj + (size_t)v * g->dvmax, g->vdeg[v], sizeof(int), cmp_int);
    for (int c = 0; c < m; c++) qsort(g->cadj + (size_t)c * g->dcmax, g->cdeg[c], sizeof(int), cmp_int);
    for (int v = 0; v < n; v++)
        for (int i = 0; i < g->vdeg[v]; i++) {
            int c = g->vadj[v * g->dvmax + i];
            int p = -1;
            for (int q = 0; q < g->cdeg[c]; q++) if (g->cadj[c * g->dcmax + q] == v) p = q;
            g->vpos[v * g->dvmax + i] = p;
        }
    free(fv); free(fc);
    return g;
}

/* Eqs. 1-2: block (i,j) with exponent a >= 0 is P^a, the identity shifted
 * right a times, i.e. row r of the block has its 1 in column (r + a) mod Z;
 * a = -1 is the zero block.  Variable node j*Z+k, check node i*Z+r. */
og_graph *og_from_qc(int m_b, int n_b, int Z, const int *shifts) {
    int E = 0;
    for (int i = 0; i < m_b * n_b; i++) if (shifts[i] >= 0) E += Z;
    int *ec = (int *)malloc(sizeof(int) * (E ? E : 1)), *ev = (int *)malloc(sizeof(int) * (E ? E : 1));
    int e = 0;
    for (int i = 0; i < m_b; i++)
        for (int j = 0; j < n_b; j++) {
            int a = shifts[i * n_b + j];
            if (a < 0) continue;
            for (int r = 0; r < Z; r++) { ec[e] = i * Z + r; ev[e] = j * Z + (r + a) % Z; e++; }
        }
    og_graph *g = graph_from_edges(n_b * Z, m_b * Z, E, ec, ev);
    g->Z = Z; g->n_b = n_b; g->m_b = m_b;
    free(ec); free(ev);
    return g;
}

/* A general parity-check matrix given by its rows (no automorphism used). */
og_graph *og_from_csr(int n, int m, const int *row_ptr, const int *col_idx) {
    int E = row_ptr[m];
    int *ec = (int *)malloc(sizeof(int) * (E ? E : 1));
    for (int c = 0; c < m; c++) for (int e = row_ptr[c]; e < row_ptr[c + 1]; e++) ec[e] = c;
    og_graph *g = graph_from_edges(n, m, E, ec, col_idx);
    free(ec);
    return g;
}

void og_free(og_graph *g) {
    if (!g) return;
    free(g->vdeg); free(g->vadj); free(g->vpos); free(g->cdeg); free(g->cadj); free(g);
}

int og_n(const og_graph *g) { return g->n; }
int og_m(const og_graph *g) { return g->m; }
int og_E(const og_graph *g) { return g->E; }
int og_vdeg(const og_graph *g, int v) { return g->vdeg[v]; }
int og_cdeg(const og_graph *g, int c) { return g->cdeg[c]; }
int og_vadj(const og_graph *g, int v, int i) { return g->vadj[v * g->dvmax + i]; }
int og_cadj(const og_graph *g, int c, int p) { return g->cadj[c * g->dcmax + p]; }

/* Girth: shortest cycle of the Tanner graph, by breadth-first search from
 * every variable node (every cycle passes through one).  Returns 0 if the
 * graph has no cycle. */
int og_girth(og_graph *g) {
    if (g->girth) return g->girth;
    int N = g->n + g->m;
    int *dist = (int *)malloc(sizeof(int) * N), *par = (int *)malloc(sizeof(int) * N);
    int *queue = (int *)malloc(sizeof(int) * N);
    int best = 1 << 30;
    for (int s = 0; s < g->n; s++) {
        for (int i = 0; i < N; i++) dist[i] = -1;
        int qh = 0, qt = 0;
        dist[s] = 0; par[s] = -1; queue[qt++] = s;
        while (qh < qt) {
            int u = queue[qh++];
            if (2 * dist[u] + 1 >= best) break;
            int deg = u < g->n ? g->vdeg[u] : g->cdeg[u - g->n];
            for (int k = 0; k < deg; k++) {
                int w = u < g->n ? g->n + g->vadj[u * g->dvmax + k] : g->cadj[(u - g->n) * g->dcmax + k];
                if (w == par[u]) continue;
                if (dist[w] < 0) { dist[w] = dist[u] + 1; par[w] = u; queue[qt++] = w; }
                else if (dist[u] + dist[w] + 1 < best) best = dist[u] + dist[w] + 1;
            }
        }
    }
    free(dist); free(par); free(queue);
    g->girth = best == (1 << 30) ? 0 : best;
    return g->girth;
}

/* Tanner ball: the variable nodes other than v reached from v along
 * VN-CN-VN or VN-CN-VN-CN-VN, i.e. the variable layers of the depth-3
 * unrolled tree VN1-CN1-VN2-CN2-VN3 of Sec. III (Fig. 3).  Ascending. */
int og_ball4(const og_graph *g, int v, int *out) {
    unsigned char *seen = (unsigned char *)calloc(g->n, 1);
    seen[v] = 1;
    int cnt = 0;
    for (int i = 0; i < g->vdeg[v]; i++) {
        int c = g->vadj[v * g->dvmax + i];
        for (int p = 0; p < g->cdeg[c]; p++) {
            int u = g->cadj[c * g->dcmax + p];
            if (!seen[u]) { seen[u] = 1; out[cnt++] = u; }
        }
    }
    int d2 = cnt;
    for (int t = 0; t < d2; t++) {
        int u = out[t];
        for (int i = 0; i < g->vdeg[u]; i++) {
            int c = g->vadj[u * g->dvmax + i];
            for (int p = 0; p < g->cdeg[c]; p++) {
                int w = g->cadj[c * g->dcmax + p];
                if (!seen[w]) { seen[w] = 1; out[cnt++] = w; }
            }
        }
    }
    free(seen);
    qsort(out, cnt, sizeof(int), cmp_int);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Cycles and their EMD (Sec. II, Table II; cycle density, Table V)     */
/* ------------------------------------------------------------------ */

/* Sec. II, Prop. 1 and Table II.  A "cycle" of length 2l is read as an
 * exponent chain that closes (eq. 3), i.e. a closed walk
 * v0 - c1 - v1 - ... - v_{l-1} - c_l - v0 of the Tanner graph that never
 * steps straight back (c_{t+1} != c_t, v_{t+1} != v_t, and c_l != c_1), taken
 * up to rotation and reversal; it may pass a node twice (the 4-cycle walked
 * twice is an 8-cycle of Table II's EMD-2 row).  Its EMD is the number of
 * check nodes connected to exactly one variable node of the walk.
 *
 * A walk class with rotation period p (smallest p with v_{t+p} = v_t and
 * c_{t+p} = c_t) has p rotations, times 2 directions unless its reverse is
 * one of them (r = 1 or 2), so it is met p r times as a walk from a start
 * node; each walk adds 2l / (p r) to hist2[l][EMD], and hist2 / (2l) summed
 * over every start node counts classes (over the orbit representatives of a
 * QC code it counts classes per circulant orbit, Table II's "without
 * multiplication by graph automorphism").  For l <= 3 every such walk is a
 * simple cycle, and walks[l] from v is twice the cycles through v. */
static int og_walk_emd(const og_graph *g, const int *vs, int L) {
    int u[16], nu = 0;
    for (int x = 0; x < L; x++) {
        int dup = 0;
        for (int y = 0; y < nu; y++) dup |= u[y] == vs[x];
        if (!dup) u[nu++] = vs[x];
    }
    int emd = 0;
    for (int x = 0; x < nu; x++)
        for (int i = 0; i < g->vdeg[u[x]]; i++) {
            int c = g->vadj[u[x] * g->dvmax + i], k = 0;
            for (int y = 0; y < nu; y++)
                for (int p = 0; p < g->cdeg[c]; p++) k += g->cadj[c * g->dcmax + p] == u[y];
            emd += k == 1;
        }
    return emd;
}

/* p r of the closed walk vs[0..L-1], cs[1..L] (cs[t] between vs[t-1] and vs[t mod L]) */
static int og_walk_reps(const int *vs, const int *cs, int L) {
    int p = L;
    for (int q = 1; q < L; q++) {
        if (L % q) continue;
        int ok = 1;
        for (int t = 0; t < L && ok; t++) ok = vs[(t + q) % L] == vs[t] && cs[(t + q) % L + 1] == cs[t + 1];
        if (ok) { p = q; break; }
    }
    /* reversed: v0, c_L, v_{L-1}, c_{L-1}, ...; rotated by s it equals the walk if
     * v_{(s-t) mod L} = v_t and the check after it, c_{(s-t) mod L} (c_0 = c_L), = c_{t+1} */
    int r = 2;
    for (int sft = 0; sft < L && r == 2; sft++) {
        int ok = 1;
        for (int t = 0; t < L && ok; t++) {
            int a = ((sft - t) % L + L) % L;
            ok = vs[a] == vs[t] && cs[a == 0 ? L : a] == cs[t + 1];
        }
        if (ok) r = 1;
    }
    return p * r;
}

static void walks_from(const og_graph *g, int lmax, int d, int *vs, int *cs, long long *walks, long long *hist2) {
    int v = vs[d];
    for (int i = 0; i < g->vdeg[v]; i++) {
        int c = g->vadj[v * g->dvmax + i];
        if (d >= 1 && c == cs[d]) continue;  /* no step straight back */
        if (d >= 1 && c != cs[1] && v != vs[0]) {
            int closes = 0;
            for (int p = 0; p < g->cdeg[c]; p++) closes |= g->cadj[c * g->dcmax + p] == vs[0];
            if (closes) {
                cs[d + 1] = c;
                walks[d + 1]++;
                if (hist2) hist2[(d + 1) * 128 + og_walk_emd(g, vs, d + 1)] += 2 * (d + 1) / og_walk_reps(vs, cs, d + 1);
            }
        }
        if (d + 1 >= lmax) continue;
        for (int p = 0; p < g->cdeg[c]; p++) {
            int u = g->cadj[c * g->dcmax + p];
            if (u == v) continue;
            cs[d + 1] = c;
            vs[d + 1] = u;
            walks_from(g, lmax, d + 1, vs, cs, walks, hist2);
        }
    }
}

/* The closed walks from v of l = 2..lmax variable nodes (as above):
 * walks[l] (lmax + 1 entries) and, if hist2 is not NULL, hist2[l * 128 + e]
 * += 2l / (p r) per walk.  Both are added to. */
void og_cycles_from(const og_graph *g, int v, int lmax, long long *walks, long long *hist2) {
    int vs[16], cs[17];
    vs[0] = v;
    walks_from(g, lmax, 0, vs, cs, walks, hist2);
}

/* ------------------------------------------------------------------ */
/* Canonical form under the circulant shift (graph automorphism)       */
/* ------------------------------------------------------------------ */

/* Shifting every variable node (j,k) to (j,(k+s) mod Z) (and every check
 * likewise) maps the QC Tanner graph onto itself (Sec. III: "graph
 * automorphism"; Table III counts are multiples of Z = 128).  The key of a
 * set T is the lexicographically smallest sorted tuple among the shifts by
 * s = -(v mod Z), v in T; a general code uses the sorted set itself.  The
 * orbit size is Z / |{s in [0,Z): T + s = T}|.  Returns the orbit size. */
static int lex_less(const int *a, const int *b, int n) {
    for (int i = 0; i < n; i++) if (a[i] != b[i]) return a[i] < b[i];
    return 0;
}

int og_canon(const og_graph *g, const int *T, int a, int *key) {
    if (a == 0) return 1;
    if (g->Z == 0) {
        memcpy(key, T, sizeof(int) * a);
        qsort(key, a, sizeof(int), cmp_int);
        return 1;
    }
    int Z = g->Z;
    int *tmp = (int *)malloc(sizeof(int) * a), *base = (int *)malloc(sizeof(int) * a);
    memcpy(base, T, sizeof(int) * a);
    qsort(base, a, sizeof(int), cmp_int);
    int have = 0;
    for (int t = 0; t < a; t++) {
        int s = (Z - T[t] % Z) % Z;
        for (int i = 0; i < a; i++) tmp[i] = (T[i] / Z) * Z + (T[i] % Z + s) % Z;
        qsort(tmp, a, sizeof(int), cmp_int);
        if (!have || lex_less(tmp, key, a)) { memcpy(key, tmp, sizeof(int) * a); have = 1; }
    }
    int stab = 0;
    for (int s = 0; s < Z; s++) {
        for (int i = 0; i < a; i++) tmp[i] = (T[i] / Z) * Z + (T[i] % Z + s) % Z;
        qsort(tmp, a, sizeof(int), cmp_int);
        if (memcmp(tmp, base, sizeof(int) * a) == 0) stab++;
    }
    free(tmp); free(base);
    return Z / stab;
}

/* ------------------------------------------------------------------ */
/* Candidate impulse sets                                              */
/* ------------------------------------------------------------------ */

/* Sec. III: for each orbit representative VN (QC: (j,0); general: every
 * VN), impulse sets are drawn from the depth-3 tree around it.  Reading:
 * a set contains the representative and at most max_size-1 other nodes of
 * its Tanner ball; with cycle_len = 2l > 0 the variable-node sets of the
 * 2l-cycles through the representative are added.  Every set is reduced to
 * its canonical key and duplicates are dropped. */
typedef struct { int size; int v[4]; } og_cand;

static int cmp_cand(const void *pa, const void *pb) {
    const og_cand *a = (const og_cand *)pa, *b = (const og_cand *)pb;
    if (a->size != b->size) return a->size < b->size ? -1 : 1;
    for (int i = 0; i < a->size; i++) if (a->v[i] != b->v[i]) return a->v[i] < b->v[i] ? -1 : 1;
    return 0;
}

typedef struct { og_cand *c; size_t n, cap; } cand_vec;

static void cv_push(const og_graph *g, cand_vec *cv, const int *vars, int size) {
    if (cv->n == cv->cap) {
        cv->cap = cv->cap ? 2 * cv->cap : 1024;
        cv->c = (og_cand *)realloc(cv->c, sizeof(og_cand) * cv->cap);
    }
    og_cand *o = &cv->c[cv->n++];
    o->size = size;
    int key[4];
    og_canon(g, vars, size, key);
    for (int i = 0; i < 4; i++) o->v[i] = i < size ? key[i] : -1;
}

/* all simple cycles of length 2l through variable node v0, as VN sets */
static void cycles_from(const og_graph *g, int v0, int l, int depth, int *vs, int *cs,
                        cand_vec *cv) {
    int v = vs[depth];
    for (int i = 0; i < g->vdeg[v]; i++) {
        int c = g->vadj[v * g->dvmax + i];
        int used = 0;
        for (int t = 0; t < depth; t++) if (cs[t] == c) used = 1;
        if (used) continue;
        for (int p = 0; p < g->cdeg[c]; p++) {
            int u = g->cadj[c * g->dcmax + p];
            if (u == v) continue;
            if (depth == l - 1) {
                if (u == v0) { cs[depth] = c; cv_push(g, cv, vs, l); }
                continue;
            }
            int dup = 0;
            for (int t = 0; t <= depth; t++) if (vs[t] == u) dup = 1;
            if (dup) continue;
            cs[depth] = c; vs[depth + 1] = u;
            cycles_from(g, v0, l, depth + 1, vs, cs, cv);
        }
    }
}

typedef struct { og_cand *c; size_t n; } og_cands;

og_cands *og_candidates(const og_graph *g, int max_size, int cycle_len) {
    cand_vec cv = {0};
    int *ball = (int *)malloc(sizeof(int) * g->n);
    int nrep = g->Z ? g->n_b : g->n;
    for (int r = 0; r < nrep; r++) {
        int v0 = g->Z ? r * g->Z : r;
        int B = og_ball4(g, v0, ball);
        int s[4] = {v0, 0, 0, 0};
        if (max_size >= 1) cv_push(g, &cv, s, 1);
        for (int i = 0; i < B && max_size >= 2; i++) {
            s[1] = ball[i];
            cv_push(g, &cv, s, 2);
            for (int j = i + 1; j < B && max_size >= 3; j++) {
                s[2] = ball[j];
                cv_push(g, &cv, s, 3);
                for (int k = j + 1; k < B && max_size >= 4; k++) { s[3] = ball[k]; cv_push(g, &cv, s, 4); }
            }
        }
        if (cycle_len >= 4 && cycle_len <= 8) {
            int vs[4] = {v0, 0, 0, 0}, cs[4];
            cycles_from(g, v0, cycle_len / 2, 0, vs, cs, &cv);
        }
    }
    free(ball);
    qsort(cv.c, cv.n, sizeof(og_cand), cmp_cand);
    size_t u = 0;
    for (size_t i = 0; i < cv.n; i++)
        if (u == 0 || cmp_cand(&cv.c[u - 1], &cv.c[i]) != 0) cv.c[u++] = cv.c[i];
    og_cands *out = (og_cands *)malloc(sizeof(og_cands));
    out->c = cv.c; out->n = u;
    return out;
}

size_t og_cands_count(const og_cands *c) { return c->n; }
void og_cands_copy(const og_cands *c, int *out /* n x 5: size, v0..v3 */) {
    for (size_t i = 0; i < c->n; i++) {
        out[5 * i] = c->c[i].size;
        for (int k = 0; k < 4; k++) out[5 * i + 1 + k] = c->c[i].v[k];
    }
}
void og_cands_free(og_cands *c) { if (c) { free(c->c); free(c); } }

/* ------------------------------------------------------------------ */
/* Decoders                                                            */
/* ------------------------------------------------------------------ */

static int clampi(int x, int lo, int hi) { return x < lo ? lo : x > hi ? hi : x; }
static float clampf(float x, float lo, float hi) { return x < lo ? lo : x > hi ? hi : x; }

static int unsat_count(const og_graph *g, const unsigned char *x) {
    int u = 0;
    for (int c = 0; c < g->m; c++) {
        int par = 0;
        for (int p = 0; p < g->cdeg[c]; p++) par ^= x[g->cadj[c * g->dcmax + p]];
        u += par;
    }
    return u;
}

/* Fixed-point normalized min-sum, flooding schedule (the decoder of the
 * enumeration is left open by the paper, Sec. III; this is the int16
 * decoder of the workload definition).
 *   start:  q(v->c) = L_v;  x_0 = [L_v < 0]
 *   check:  r(c->v) = s * ((an * m) >> as), m = min over v' != v of |q(v'->c)|,
 *           s = product over v' != v of sgn q(v'->c), sgn(0) = +1
 *   var:    P_v = L_v + sum_c r(c->v);  q(v->c) = clamp(P_v - r(c->v), -sat, sat);
 *           x_v = [P_v < 0]
 *   u_k = number of unsatisfied checks of x_k (w_H(H x_k), Sec. III); stop at
 *   the first k with u_k = 0, else after K iterations (K_last = k).
 * Best error pattern (Sec. III, S(min_iter w_H(H x_iter)) with the list
 * starting at x_{floor(girth/2)}): x* = x_k for the first k in
 * [wstart, K_last] with minimal u_k; if K_last < wstart, x* = x_{K_last}.
 * Returns 1 if the decoder failed (x_{K_last} != 0), else 0.  x_trace, when
 * given, receives every x_k, k = 0..K_last. */
int og_decode_nms(const og_graph *g, const int *L, int K, int sat, int an, int as, int wstart,
                  unsigned char *xbest, int *K_last, int *u_trace /* K+1 or NULL */,
                  int *P_out /* n or NULL: P_v after the last iteration run */,
                  unsigned char *x_trace /* (K+1) x n or NULL: x_k in row k */) {
    int E = g->m * g->dcmax;
    int *q = (int *)malloc(sizeof(int) * E), *r = (int *)malloc(sizeof(int) * E);
    unsigned char *x = (unsigned char *)malloc(g->n);
    for (int v = 0; v < g->n; v++) {
        if (P_out) P_out[v] = L[v];
        x[v] = L[v] < 0;
        for (int i = 0; i < g->vdeg[v]; i++)
            q[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]] = L[v];
    }
    int u = unsat_count(g, x), ubest = 1 << 30, kl = 0;
    if (u_trace) u_trace[0] = u;
    if (x_trace) memcpy(x_trace, x, g->n);
    for (int k = 1; k <= K && u != 0; k++) {
        for (int c = 0; c < g->m; c++) {
            int d = g->cdeg[c];
            for (int p = 0; p < d; p++) {
                int mn = 1 << 30, sg = 1;
                for (int p2 = 0; p2 < d; p2++) {
                    if (p2 == p) continue;
                    int qq = q[c * g->dcmax + p2];
                    int mag = qq < 0 ? -qq : qq;
                    if (mag < mn) mn = mag;
                    if (qq < 0) sg = -sg;
                }
                if (d == 1) mn = sat; /* no other edge: the check alone forces 0 */
                r[c * g->dcmax + p] = sg * ((an * mn) >> as);
            }
        }
        for (int v = 0; v < g->n; v++) {
            int P = L[v];
            for (int i = 0; i < g->vdeg[v]; i++)
                P += r[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]];
            for (int i = 0; i < g->vdeg[v]; i++) {
                int e = g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i];
                q[e] = clampi(P - r[e], -sat, sat);
            }
            x[v] = P < 0;
            if (P_out) P_out[v] = P;
        }
        u = unsat_count(g, x);
        if (u_trace) u_trace[k] = u;
        if (x_trace) memcpy(x_trace + (size_t)k * g->n, x, g->n);
        kl = k;
        if (k >= wstart && u < ubest) { ubest = u; memcpy(xbest, x, g->n); }
    }
    if (kl < wstart) memcpy(xbest, x, g->n);
    int fail = 0;
    for (int v = 0; v < g->n; v++) fail |= x[v];
    *K_last = kl;
    free(q); free(r); free(x);
    return fail;
}

/* The simulation decoder of Sec. III (the FER curves of Fig. 2): quantized
 * normalized layered min-sum, LLR 4 bits, check-to-variable 4 bits,
 * variable-to-check 6 bits, 20 iterations.  The paper names the widths and
 * nothing else; readings:
 *   - every quantity is a signed integer; a w-bit value saturates to
 *     +-(2^(w-1) - 1); the channel LLR L_v is saturated to the LLR width;
 *   - a layer is a row block of the QC base matrix (whose checks touch
 *     distinct variable nodes), for a general code one check row, in order;
 *   - the posterior P_v (start: L_v) is kept at the variable-to-check width;
 *   - one layer: for every edge (c, v) of the layer, from the P_v before the
 *     layer, q = sat_v2c(P_v - r(c,v)); then for every check of the layer
 *     r(c,v) = s * sat_c2v((an * m) >> as), m = min over v' != v of |q(c,v')|
 *     (sat_c2v when c has no other edge), s = product of their signs
 *     (sgn 0 = +1); then P_v = sat_v2c(q(c,v) + r(c,v));
 *   - after each full iteration x_v = [P_v < 0], u = unsatisfied checks; stop
 *     at u = 0 (also before the first iteration) or after K iterations.
 * Returns 1 if x != 0 at the end; x_out receives x, *K_last the iterations run. */
static int satw(int x, int w) {
    const int lim = (1 << (w - 1)) - 1;
    return x < -lim ? -lim : x > lim ? lim : x;
}
int og_decode_lnms(const og_graph *g, const int *L, int K, int llr_bits, int c2v_bits, int v2c_bits, int an,
                   int as, unsigned char *x_out, int *K_last) {
    const int E = g->m * g->dcmax;
    int *r = (int *)calloc((size_t)E, sizeof(int)), *q = (int *)malloc(sizeof(int) * E);
    int *P = (int *)malloc(sizeof(int) * g->n);
    unsigned char *x = (unsigned char *)malloc(g->n);
    for (int v = 0; v < g->n; v++) { P[v] = satw(L[v], llr_bits); x[v] = P[v] < 0; }
    const int layer = g->Z > 0 ? g->Z : 1;   /* checks per layer */
    const int nl = g->m / layer;
    int u = unsat_count(g, x), kl = 0;
    for (int k = 1; k <= K && u != 0; k++) {
        for (int l = 0; l < nl; l++) {
            const int c0 = l * layer, c1 = c0 + layer;
            for (int c = c0; c < c1; c++)
                for (int p = 0; p < g->cdeg[c]; p++) {
                    const int e = c * g->dcmax + p;
                    q[e] = satw(P[g->cadj[e]] - r[e], v2c_bits);
                }
            for (int c = c0; c < c1; c++) {
                const int d = g->cdeg[c];
                for (int p = 0; p < d; p++) {
                    int mn = 1 << 30, sg = 1;
                    for (int p2 = 0; p2 < d; p2++) {
                        if (p2 == p) continue;
                        const int qq = q[c * g->dcmax + p2];
                        const int mag = qq < 0 ? -qq : qq;
                        if (mag < mn) mn = mag;
                        if (qq < 0) sg = -sg;
                    }
                    const int mag = d == 1 ? (1 << (c2v_bits - 1)) - 1 : satw((an * mn) >> as, c2v_bits);
                    r[c * g->dcmax + p] = sg * mag;
                }
            }
            for (int c = c0; c < c1; c++)
                for (int p = 0; p < g->cdeg[c]; p++) {
                    const int e = c * g->dcmax + p;
                    P[g->cadj[e]] = satw(q[e] + r[e], v2c_bits);
                }
        }
        for (int v = 0; v < g->n; v++) x[v] = P[v] < 0;
        u = unsat_count(g, x);
        kl = k;
    }
    int fail = 0;
    for (int v = 0; v < g->n; v++) fail |= x[v];
    if (x_out) memcpy(x_out, x, g->n);
    *K_last = kl;
    free(r); free(q); free(P); free(x);
    return fail;
}

/* Single-precision tanh and atanh used by the sum-product decoder, from
 * their series with every operation an IEEE single-precision add, multiply
 * or divide (no fused multiply-add; ldexpf/frexpf/rintf are exact), so that
 * any implementation taking the same steps gets the same bits:
 *   expm1(x), x >= 0: k = rint(x / ln2), r = (x - k ln2_hi) - k ln2_lo
 *     (Cody-Waite reduction), expm1(r) = r + r^2/2! + ... + r^9/9! by
 *     Horner, expm1(x) = 2^k (expm1(r) + 1) - 1 for k != 0;
 *   tanh(y) = sgn(y) e/(e + 2), e = expm1(2|y|);
 *   atanh(p) = sgn(p) (a + a^3/3 + ... + a^17/17) for a = |p| < 1/4,
 *     else sgn(p) log(t)/2 with t = (1 + a)/(1 - a), t = m 2^e, m in
 *     [sqrt(1/2), sqrt(2)), log t = e ln2 + 2 (s + s^3/3 + ... + s^13/13),
 *     s = (m - 1)/(m + 1). */
static const float OG_LN2_HI = 0.693145751953125f;
static const float OG_LN2_LO = 1.42860676533018704e-06f;
static const float OG_INV_LN2 = 1.44269504088896341f;
static const float OG_LN2 = 0.693147180559945309f;
static const float OG_SQRT_HALF = 0.707106781186547524f;

static float og_expm1_pos(float x) {
    float k = rintf(x * OG_INV_LN2);
    float r = (x - k * OG_LN2_HI) - k * OG_LN2_LO;
    float p = 1.0f / 362880.0f;
    p = p * r + 1.0f / 40320.0f;
    p = p * r + 1.0f / 5040.0f;
    p = p * r + 1.0f / 720.0f;
    p = p * r + 1.0f / 120.0f;
    p = p * r + 1.0f / 24.0f;
    p = p * r + 1.0f / 6.0f;
    p = p * r + 0.5f;
    p = p * r + 1.0f;
    p = p * r;
    if (k == 0.0f) return p;
    return ldexpf(p + 1.0f, (int)k) - 1.0f;
}

float og_tanhf(float y) {
    float a = fabsf(y);
    float e = og_expm1_pos(a + a);
    float t = e / (e + 2.0f);
    return y < 0.0f ? -t : t;
}

float og_atanhf(float p) {
    float a = fabsf(p), r;
    if (a < 0.25f) {
        float a2 = a * a;
        float q = 1.0f / 17.0f;
        q = q * a2 + 1.0f / 15.0f;
        q = q * a2 + 1.0f / 13.0f;
        q = q * a2 + 1.0f / 11.0f;
        q = q * a2 + 1.0f / 9.0f;
        q = q * a2 + 1.0f / 7.0f;
        q = q * a2 + 1.0f / 5.0f;
        q = q * a2 + 1.0f / 3.0f;
        q = q * a2 + 1.0f;
        r = q * a;
    } else {
        float t = (1.0f + a) / (1.0f - a);
        int e;
        float m = frexpf(t, &e);
        if (m < OG_SQRT_HALF) { m = m + m; e = e - 1; }
        float s = (m - 1.0f) / (m + 1.0f);
        float s2 = s * s;
        float q = 1.0f / 13.0f;
        q = q * s2 + 1.0f / 11.0f;
        q = q * s2 + 1.0f / 9.0f;
        q = q * s2 + 1.0f / 7.0f;
        q = q * s2 + 1.0f / 5.0f;
        q = q * s2 + 1.0f / 3.0f;
        q = q * s2 + 1.0f;
        float lg = (float)e * OG_LN2 + (s + s) * q;
        r = 0.5f * lg;
    }
    return p < 0.0f ? -r : r;
}

/* Floating-point sum-product (same flooding schedule and stopping rule).
 *   check:  r(c->v) = 2 atanh( prod over v' != v, ascending, of tanh(q(v'->c)/2) ),
 *           with og_tanhf / og_atanhf above,
 *           +-clip when |prod| >= 1, then clipped to [-clip, clip]
 *   var:    P_v = L_v + r(c_0->v) + r(c_1->v) + ... (checks ascending);
 *           q(v->c) = clip(P_v - r(c->v)); x_v = [P_v < 0]
 * Single precision, as the workload states. */
/* libm = 1: the check update uses the C library's tanhf / atanhf instead of
 * the series above (the other reading of the single-precision decoder: any
 * correctly implemented tanh/atanh; thresholds then agree within the stated
 * tolerance rather than bit for bit). */
static float spa_tanh(float x, int libm) { return libm ? tanhf(x) : og_tanhf(x); }
static float spa_atanh(float x, int libm) { return libm ? atanhf(x) : og_atanhf(x); }

int og_decode_spa(const og_graph *g, const float *L, int K, float clip, int wstart,
                  unsigned char *xbest, int *K_last, int *u_trace, int libm) {
    int E = g->m * g->dcmax;
    float *q = (float *)malloc(sizeof(float) * E), *r = (float *)malloc(sizeof(float) * E);
    float *t = (float *)malloc(sizeof(float) * g->dcmax);
    unsigned char *x = (unsigned char *)malloc(g->n);
    for (int v = 0; v < g->n; v++) {
        x[v] = L[v] < 0.0f;
        for (int i = 0; i < g->vdeg[v]; i++)
            q[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]] = L[v];
    }
    int u = unsat_count(g, x), ubest = 1 << 30, kl = 0;
    if (u_trace) u_trace[0] = u;
    for (int k = 1; k <= K && u != 0; k++) {
        for (int c = 0; c < g->m; c++) {
            int d = g->cdeg[c];
            for (int p = 0; p < d; p++) t[p] = spa_tanh(q[c * g->dcmax + p] * 0.5f, libm);
            for (int p = 0; p < d; p++) {
                float prod = 1.0f;
                for (int p2 = 0; p2 < d; p2++) if (p2 != p) prod = prod * t[p2];
                float rr;
                if (fabsf(prod) >= 1.0f) rr = prod > 0.0f ? clip : -clip;
                else rr = 2.0f * spa_atanh(prod, libm);
                r[c * g->dcmax + p] = clampf(rr, -clip, clip);
            }
        }
        for (int v = 0; v < g->n; v++) {
            float P = L[v];
            for (int i = 0; i < g->vdeg[v]; i++)
                P = P + r[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]];
            for (int i = 0; i < g->vdeg[v]; i++) {
                int e = g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i];
                q[e] = clampf(P - r[e], -clip, clip);
            }
            x[v] = P < 0.0f;
        }
        u = unsat_count(g, x);
        if (u_trace) u_trace[k] = u;
        kl = k;
        if (k >= wstart && u < ubest) { ubest = u; memcpy(xbest, x, g->n); }
    }
    if (kl < wstart) memcpy(xbest, x, g->n);
    int fail = 0;
    for (int v = 0; v < g->n; v++) fail |= x[v];
    *K_last = kl;
    free(q); free(r); free(t); free(x);
    return fail;
}

/* Exact posterior-LLR sum-product output on the final iteration, for
 * tests on cycle-free codes: returns P_v after exactly K iterations
 * without early stopping. */
void og_spa_posterior(const og_graph *g, const float *L, int K, float clip, float *P_out) {
    int E = g->m * g->dcmax;
    float *q = (float *)malloc(sizeof(float) * E), *r = (float *)malloc(sizeof(float) * E);
    float *t = (float *)malloc(sizeof(float) * g->dcmax);
    for (int v = 0; v < g->n; v++) {
        P_out[v] = L[v];
        for (int i = 0; i < g->vdeg[v]; i++)
            q[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]] = L[v];
    }
    for (int k = 1; k <= K; k++) {
        for (int c = 0; c < g->m; c++) {
            int d = g->cdeg[c];
            for (int p = 0; p < d; p++) t[p] = og_tanhf(q[c * g->dcmax + p] * 0.5f);
            for (int p = 0; p < d; p++) {
                float prod = 1.0f;
                for (int p2 = 0; p2 < d; p2++) if (p2 != p) prod = prod * t[p2];
                float rr;
                if (fabsf(prod) >= 1.0f) rr = prod > 0.0f ? clip : -clip;
                else rr = 2.0f * og_atanhf(prod);
                r[c * g->dcmax + p] = clampf(rr, -clip, clip);
            }
        }
        for (int v = 0; v < g->n; v++) {
            float P = L[v];
            for (int i = 0; i < g->vdeg[v]; i++)
                P = P + r[g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i]];
            for (int i = 0; i < g->vdeg[v]; i++) {
                int e = g->vadj[v * g->dvmax + i] * g->dcmax + g->vpos[v * g->dvmax + i];
                q[e] = clampf(P - r[e], -clip, clip);
            }
            P_out[v] = P;
        }
    }
    free(q); free(r); free(t);
}

/* ------------------------------------------------------------------ */
/* Trapping-set extraction (Sec. III, S1/S2 sieving)                   */
/* ------------------------------------------------------------------ */

/* |N(c) cap S| for the indicator S */
static int check_count(const og_graph *g, int c, const unsigned char *S) {
    int k = 0;
    for (int p = 0; p < g->cdeg[c]; p++) k += S[g->cadj[c * g->dcmax + p]];
    return k;
}

/* Tree(S): the largest subset of S whose induced subgraph has no tree-like
 * part, i.e. the variable nodes of the 2-core of the bipartite graph on S
 * and N(S): checks with at most one neighbour in the set and variable nodes
 * with at most one remaining check are deleted until none is left.  In place. */
void og_tree(const og_graph *g, unsigned char *S) {
    int changed = 1;
    while (changed) {
        changed = 0;
        for (int v = 0; v < g->n; v++) {
            if (!S[v]) continue;
            int live = 0;
            for (int i = 0; i < g->vdeg[v]; i++)
                if (check_count(g, g->vadj[v * g->dvmax + i], S) >= 2) live++;
            if (live < 2) { S[v] = 0; changed = 1; }
        }
    }
}

/* TS(S): S together with every variable node outside S that has at least
 * two checks in N(S), i.e. closes a new cycle with S (one pass). */
void og_ts_closure(const og_graph *g, const unsigned char *S, unsigned char *out) {
    unsigned char *inN = (unsigned char *)calloc(g->m, 1);
    for (int c = 0; c < g->m; c++) inN[c] = check_count(g, c, S) >= 1;
    for (int v = 0; v < g->n; v++) {
        out[v] = S[v];
        if (S[v]) continue;
        int k = 0;
        for (int i = 0; i < g->vdeg[v]; i++) k += inN[g->vadj[v * g->dvmax + i]];
        if (k >= 2) out[v] = 1;
    }
    free(inN);
}

/* TS(a,b) of Sec. II: a = |T|, b = number of checks with an odd number of
 * neighbours in T.  *elem = 1 if every check touching T touches it at most
 * twice (an elementary set). */
void og_classify(const og_graph *g, const unsigned char *T, int *a, int *b, int *elem) {
    int aa = 0, bb = 0, el = 1;
    for (int v = 0; v < g->n; v++) aa += T[v];
    for (int c = 0; c < g->m; c++) {
        int k = check_count(g, c, T);
        if (k & 1) bb++;
        if (k > 2) el = 0;
    }
    *a = aa; *b = bb; *elem = el;
}

/* Sieving (Sec. III): with X = supp(x*) cup I, take S1 = Tree(X) if it is
 * not empty, else S2 = Tree(TS(X)).  Returns 1 (S1), 2 (S2) or 0 (both
 * empty: an acyclic failure, not a trapping set).  T receives the set. */
int og_extract(const og_graph *g, const unsigned char *xstar, const int *I, int nI,
               unsigned char *T) {
    unsigned char *X = (unsigned char *)malloc(g->n);
    memcpy(X, xstar, g->n);
    for (int t = 0; t < nI; t++) X[I[t]] = 1;
    memcpy(T, X, g->n);
    og_tree(g, T);
    int which = 1, any = 0;
    for (int v = 0; v < g->n; v++) any |= T[v];
    if (!any) {
        og_ts_closure(g, X, T);
        og_tree(g, T);
        which = 2;
        any = 0;
        for (int v = 0; v < g->n; v++) any |= T[v];
        if (!any) which = 0;
    }
    free(X);
    return which;
}

/* ------------------------------------------------------------------ */
/* The enumeration: impulse, bisection, extraction, canonical dedupe    */
/* ------------------------------------------------------------------ */

typedef struct {
    int decoder;    /* 0 = fixed-point min-sum, 1 = float sum-product */
    int K;
    int base_llr;   /* fixed point, units of 1/8 */
    int sat;        /* fixed-point message and channel saturation */
    int alpha_num, alpha_shift;
    int amp_steps;  /* s */
    float spa_clip; /* sum-product clip */
    float spa_amax; /* sum-product: amplitude range in LLR units */
    int list_mode;  /* 1: every set of the ordered list S1(x_k), S2(x_k), k = kstart..K_last */
    int kstart;     /* first iteration of that list; 0 = floor(girth / 2) (at least 1) */
    int spa_libm;   /* sum-product with the C library's tanhf / atanhf */
    int budget_wref, budget_kmin; /* cycle-density iteration budget (wref 0 = off) */
} og_params;

typedef struct {
    int a, b, orbit, elem, count, kind;
    int thr;        /* min threshold (fixed point) */
    float thr_f;    /* min threshold (float) */
    int *key;
} og_ts;

typedef struct {
    /* per candidate */
    size_t ncand;
    int *thr;       /* -1 = no failure up to the largest amplitude */
    float *thr_f;
    int *ts;        /* index into the sorted TS list, -1 if none */
    int *which;     /* 0 none / acyclic, 1 = S1, 2 = S2 */
    int *decodes, *iters;
    /* distinct trapping sets sorted by (a, b, key) */
    int nts;
    og_ts *list;
    /* decodes that converged to the all-zero word and their iterations; the
     * first iteration of the lists in list mode */
    long long ok_decodes, ok_iters;
    int kstart_used;
} og_result;

typedef struct { int a, b, orbit, elem, kind, thr, cand; float thr_f; int *key; } ts_hit;

static int cmp_hit(const void *pa, const void *pb) {
    const ts_hit *x = (const ts_hit *)pa, *y = (const ts_hit *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    for (int i = 0; i < x->a; i++) if (x->key[i] != y->key[i]) return x->key[i] < y->key[i] ? -1 : 1;
    return 0;
}

/* The impulse of Sec. III: the impulse nodes get h(1 - eps) and all others
 * keep h.  Reading: in fixed point L_v = sat(base - A) on I and base
 * elsewhere, A = eps * h in units of 1/8; in float L_v = clip(base/8 -
 * eps * amax) on I.  The amplitude is bisected: A = 2^s - 1 first (no
 * failure there means no threshold), then up to s halvings of [lo, hi]
 * keeping the failing end; the threshold is the final hi and the trapping
 * set comes from the decode at that hi. */
static og_result *og_enumerate_stage(og_graph *g, const og_params *pp, const int *cands, size_t ncand);
void og_res_free(og_result *R);

/* Iteration budgets (Sec. III: the number of iterations varied with the
 * density of cycles through the symbol nodes; short-cycle trapping sets fail
 * within fewer iterations).  Reading: candidate I gets
 *   K(I) = kmin + ceil((K - kmin) * wref / (wref + W(I))),
 *   W(I) = sum over v in I of 2 c4(v) + c6(v),
 * c4(v) / c6(v) the 4- / 6-cycles through v (Table V's quantities per node);
 * wref = 0 gives every candidate K. */
static int *og_cycle_weights(const og_graph *g) {
    int *w = (int *)malloc(sizeof(int) * g->n);
    for (int v = 0; v < g->n; v++) {
        long long walks[4] = {0, 0, 0, 0};
        og_cycles_from(g, v, 3, walks, NULL);
        /* a cycle through v is walked twice: 2 c4 + c6 = walks4 + walks6 / 2 */
        w[v] = (int)(walks[2] + walks[3] / 2);
    }
    return w;
}

/* The enumeration.  In list mode with kstart = -1 it runs in two stages, as
 * the paper's scheduler does: first the impulse decodes of every candidate
 * (which gives the average iteration count of the decodes that converged),
 * then the ordered lists from iteration ceil(average) on. */
og_result *og_enumerate(og_graph *g, const og_params *pp, const int *cands /* ncand x 5 */,
                        size_t ncand) {
    if (!(pp->list_mode && pp->kstart < 0)) return og_enumerate_stage(g, pp, cands, ncand);
    og_params q = *pp;
    q.list_mode = 0;
    q.kstart = 0;
    og_result *first = og_enumerate_stage(g, &q, cands, ncand);
    int girth = og_girth(g), ks = girth / 2 > 1 ? girth / 2 : 1;
    if (first->ok_decodes > 0) ks = (int)((first->ok_iters + first->ok_decodes - 1) / first->ok_decodes);
    if (ks < 1) ks = 1;
    og_res_free(first);
    q = *pp;
    q.kstart = ks;
    og_result *R = og_enumerate_stage(g, &q, cands, ncand);
    R->kstart_used = ks;
    return R;
}

static og_result *og_enumerate_stage(og_graph *g, const og_params *pp, const int *cands, size_t ncand) {
    int girth = og_girth(g);
    int wstart = girth / 2 > 1 ? girth / 2 : 1;
    int *vw = pp->budget_wref > 0 ? og_cycle_weights(g) : NULL;
    long long ok = 0, okit = 0;
    og_result *R = (og_result *)calloc(1, sizeof(og_result));
    R->ncand = ncand;
    R->thr = (int *)malloc(sizeof(int) * ncand);
    R->thr_f = (float *)malloc(sizeof(float) * ncand);
    R->ts = (int *)malloc(sizeof(int) * ncand);
    R->which = (int *)malloc(sizeof(int) * ncand);
    R->decodes = (int *)malloc(sizeof(int) * ncand);
    R->iters = (int *)malloc(sizeof(int) * ncand);
    ts_hit *hits = (ts_hit *)malloc(sizeof(ts_hit) * (ncand ? ncand : 1));  /* grows in list mode */
    size_t nh = 0;
    int *Li = (int *)malloc(sizeof(int) * g->n);
    float *Lf = (float *)malloc(sizeof(float) * g->n);
    unsigned char *xb = (unsigned char *)malloc(g->n), *keep = (unsigned char *)malloc(g->n);
    unsigned char *T = (unsigned char *)malloc(g->n);
    int *tv = (int *)malloc(sizeof(int) * g->n);
    /* ordered-list mode (min-sum only): the x_k of the decode at the threshold */
    const int list = pp->list_mode && pp->decoder == 0;
    const int ks = pp->kstart > 0 ? pp->kstart : wstart;
    unsigned char *trace = list ? (unsigned char *)malloc((size_t)(pp->K + 1) * g->n) : NULL;
    unsigned char *trace_keep = list ? (unsigned char *)malloc((size_t)(pp->K + 1) * g->n) : NULL;
    unsigned char *X = (unsigned char *)malloc(g->n);
    size_t hcap = ncand ? ncand : 1;
    for (size_t ci = 0; ci < ncand; ci++) {
        int nI = cands[5 * ci];
        const int *I = cands + 5 * ci + 1;
        int decodes = 0, iters = 0, kl, failed = 0, kl_keep = 0;
        int thr = -1;
        float thr_f = -1.0f;
        int Kc = pp->K;
        if (vw) {
            long long W = 0;
            for (int t = 0; t < nI; t++) W += vw[I[t]];
            long long den = (long long)pp->budget_wref + W;
            Kc = pp->budget_kmin + (int)(((long long)(pp->K - pp->budget_kmin) * pp->budget_wref + den - 1) / den);
        }
        if (pp->decoder == 0) {
            int lo = 0, hi = (1 << pp->amp_steps) - 1;
            for (int v = 0; v < g->n; v++) Li[v] = clampi(pp->base_llr, -pp->sat, pp->sat);
            for (int t = 0; t < nI; t++) Li[I[t]] = clampi(pp->base_llr - hi, -pp->sat, pp->sat);
            int f = og_decode_nms(g, Li, Kc, pp->sat, pp->alpha_num, pp->alpha_shift, wstart, xb, &kl, NULL, NULL,
                                  list ? trace : NULL);
            decodes++; iters += kl;
            if (!f) { ok++; okit += kl; }
            if (f) {
                failed = 1; memcpy(keep, xb, g->n);
                if (list) { memcpy(trace_keep, trace, (size_t)(kl + 1) * g->n); kl_keep = kl; }
                for (int st = 0; st < pp->amp_steps && hi - lo > 1; st++) {
                    int mid = (lo + hi) >> 1;
                    for (int t = 0; t < nI; t++) Li[I[t]] = clampi(pp->base_llr - mid, -pp->sat, pp->sat);
                    f = og_decode_nms(g, Li, Kc, pp->sat, pp->alpha_num, pp->alpha_shift, wstart, xb, &kl, NULL,
                                      NULL, list ? trace : NULL);
                    decodes++; iters += kl;
                    if (!f) { ok++; okit += kl; }
                    if (f) {
                        hi = mid; memcpy(keep, xb, g->n);
                        if (list) { memcpy(trace_keep, trace, (size_t)(kl + 1) * g->n); kl_keep = kl; }
                    } else lo = mid;
                }
                thr = hi;
            }
        } else {
            float lo = 0.0f, hi = 1.0f, base = (float)pp->base_llr / 8.0f;
            for (int v = 0; v < g->n; v++) Lf[v] = clampf(base, -pp->spa_clip, pp->spa_clip);
            for (int t = 0; t < nI; t++) Lf[I[t]] = clampf(base - hi * pp->spa_amax, -pp->spa_clip, pp->spa_clip);
            int f = og_decode_spa(g, Lf, Kc, pp->spa_clip, wstart, xb, &kl, NULL, pp->spa_libm);
            decodes++; iters += kl;
            if (!f) { ok++; okit += kl; }
            if (f) {
                failed = 1; memcpy(keep, xb, g->n);
                for (int st = 0; st < pp->amp_steps; st++) {
                    float mid = 0.5f * (lo + hi);
                    for (int t = 0; t < nI; t++) Lf[I[t]] = clampf(base - mid * pp->spa_amax, -pp->spa_clip, pp->spa_clip);
                    f = og_decode_spa(g, Lf, Kc, pp->spa_clip, wstart, xb, &kl, NULL, pp->spa_libm);
                    decodes++; iters += kl;
                    if (!f) { ok++; okit += kl; }
                    if (f) { hi = mid; memcpy(keep, xb, g->n); } else lo = mid;
                }
                thr_f = hi;
            }
        }
        R->thr[ci] = thr; R->thr_f[ci] = thr_f;
        R->decodes[ci] = decodes; R->iters[ci] = iters;
        R->ts[ci] = -1; R->which[ci] = 0;
        if (!failed) continue;
        int which = og_extract(g, keep, I, nI, T);
        R->which[ci] = which;
        if (list) {
            /* Sec. III, ordered list: S1(x_k), S2(x_k) for k = kstart..K_last with
             * X_k = supp(x_k) cup I, S1 = Tree(X_k), S2 = Tree(TS(X_k)); every
             * non-empty element is a trapping set (counted once per candidate) */
            size_t first = nh;
            for (int k = ks; k <= kl_keep; k++) {
                memcpy(X, trace_keep + (size_t)k * g->n, g->n);
                for (int t = 0; t < nI; t++) X[I[t]] = 1;
                for (int part = 1; part <= 2; part++) {
                    if (part == 1) { memcpy(T, X, g->n); og_tree(g, T); }
                    else { og_ts_closure(g, X, T); og_tree(g, T); }
                    int a = 0, b, el;
                    for (int v = 0; v < g->n; v++) if (T[v]) tv[a++] = v;
                    if (!a) continue;
                    og_classify(g, T, &a, &b, &el);
                    int *key = (int *)malloc(sizeof(int) * a);
                    int orbit = og_canon(g, tv, a, key);
                    size_t dup = nh;
                    for (size_t q = first; q < nh; q++)
                        if (hits[q].a == a && !memcmp(hits[q].key, key, sizeof(int) * a)) { dup = q; break; }
                    if (dup < nh) { hits[dup].kind |= part; free(key); continue; }
                    if (nh == hcap) { hcap *= 2; hits = (ts_hit *)realloc(hits, sizeof(ts_hit) * hcap); }
                    ts_hit *h = &hits[nh++];
                    h->a = a; h->b = b; h->elem = el; h->kind = part; h->thr = thr; h->thr_f = thr_f;
                    h->cand = (int)ci; h->key = key; h->orbit = orbit;
                }
            }
            continue;
        }
        if (!which) continue;
        int a = 0, b, el;
        for (int v = 0; v < g->n; v++) if (T[v]) tv[a++] = v;
        og_classify(g, T, &a, &b, &el);
        ts_hit *h = &hits[nh++];
        h->a = a; h->b = b; h->elem = el; h->kind = which; h->thr = thr; h->thr_f = thr_f;
        h->cand = (int)ci;
        h->key = (int *)malloc(sizeof(int) * a);
        h->orbit = og_canon(g, tv, a, h->key);
    }
    qsort(hits, nh, sizeof(ts_hit), cmp_hit);
    R->list = (og_ts *)malloc(sizeof(og_ts) * (nh ? nh : 1));
    int nts = 0;
    size_t head = 0; /* first hit of the current group */
    for (size_t i = 0; i < nh; i++) {
        if (nts == 0 || cmp_hit(&hits[i], &hits[head]) != 0) {
            head = i;
            og_ts *t = &R->list[nts++];
            t->a = hits[i].a; t->b = hits[i].b; t->orbit = hits[i].orbit; t->elem = hits[i].elem;
            t->kind = hits[i].kind; t->count = 0; t->thr = hits[i].thr; t->thr_f = hits[i].thr_f;
            t->key = hits[i].key;
        }
        og_ts *t = &R->list[nts - 1];
        t->count++;
        if (hits[i].thr < t->thr) t->thr = hits[i].thr;
        if (hits[i].thr_f < t->thr_f) t->thr_f = hits[i].thr_f;
        if (list) t->kind |= hits[i].kind;
        else R->ts[hits[i].cand] = nts - 1;
    }
    for (size_t i = 0, k = 0; i < nh; i++) { /* free the keys not kept in the list */
        if (k < (size_t)nts && R->list[k].key == hits[i].key) { k++; continue; }
        free(hits[i].key);
    }
    R->nts = nts;
    R->ok_decodes = ok;
    R->ok_iters = okit;
    R->kstart_used = list ? ks : 0;
    free(hits); free(Li); free(Lf); free(xb); free(keep); free(T); free(tv);
    free(trace); free(trace_keep); free(X); free(vw);
    return R;
}

int og_res_nts(const og_result *R) { return R->nts; }
/* ok_decodes, ok_iters, kstart_used */
void og_res_stats(const og_result *R, long long *out) {
    out[0] = R->ok_decodes; out[1] = R->ok_iters; out[2] = R->kstart_used;
}
void og_res_cand(const og_result *R, int *thr, float *thr_f, int *ts, int *which, int *decodes, int *iters) {
    memcpy(thr, R->thr, sizeof(int) * R->ncand);
    memcpy(thr_f, R->thr_f, sizeof(float) * R->ncand);
    memcpy(ts, R->ts, sizeof(int) * R->ncand);
    memcpy(which, R->which, sizeof(int) * R->ncand);
    memcpy(decodes, R->decodes, sizeof(int) * R->ncand);
    memcpy(iters, R->iters, sizeof(int) * R->ncand);
}
/* info: a, b, orbit, elem, count, thr, kind; returns a */
int og_res_ts(const og_result *R, int i, int *info, float *thr_f, int *key) {
    const og_ts *t = &R->list[i];
    info[0] = t->a; info[1] = t->b; info[2] = t->orbit; info[3] = t->elem;
    info[4] = t->count; info[5] = t->thr; info[6] = t->kind;
    *thr_f = t->thr_f;
    if (key) memcpy(key, t->key, sizeof(int) * t->a);
    return t->a;
}
void og_res_free(og_result *R) {
    if (!R) return;
    for (int i = 0; i < R->nts; i++) free(R->list[i].key);
    free(R->list); free(R->thr); free(R->thr_f); free(R->ts); free(R->which);
    free(R->decodes); free(R->iters); free(R);
}

/* ------------------------------------------------------------------ */
/* Importance-sampling FER toward a trapping set                        */
/* ------------------------------------------------------------------ */
/* Sec. II-III name Cole's weighting of trapping sets by importance
 * sampling without a formula; the definition used here is mean-shift
 * importance sampling of BPSK over AWGN toward the set T:
 *   sigma^2 = 1 / (2 R Eb/N0); noise n_v = sigma g_v, g_v ~ N(0,1);
 *   y_v = 1 + n_v - mu [v in T]; channel LLR 2 y_v / sigma^2, quantized as
 *   round-half-away(8 * LLR) saturated to +-sat; decoded by the min-sum
 *   decoder from the all-zero codeword; fail = decoder failure;
 *   log w = sum_{v in T, ascending} (n_v mu / sigma^2 - mu^2 / (2 sigma^2))
 *   (the likelihood ratio of the shifted Gaussian, in double precision);
 *   FER = mean(fail * w).
 * Noise: g_v from Philox4x32-10 (Salmon et al., SC'11) with key (job low,
 * job high) and counter (v / 4, sample low, sample high, 0); its four
 * outputs x_0..x_3 become uniforms u = (2 (x >> 9) + 1) 2^-24 and two
 * Box-Muller pairs (Box and Muller 1958) (u_0,u_1) -> g_{4q}, g_{4q+1} and
 * (u_2,u_3) -> g_{4q+2}, g_{4q+3}: r = sqrt(-2 ln u_a), g = r cos(2 pi u_b),
 * g' = r sin(2 pi u_b), in single precision with IEEE-rounded operations:
 * ln by frexp and the atanh series of log, sin/cos of 2 pi u by quadrant
 * reduction and their Taylor series on [0, pi/4]. */

static void og_philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

void og_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    og_philox(c, key[0], key[1]);
    memcpy(out, c, sizeof(c));
}

float og_logf(float u) {
    int e;
    float m = frexpf(u, &e);
    if (m < OG_SQRT_HALF) { m = m + m; e = e - 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float q = 1.0f / 13.0f;
    q = q * s2 + 1.0f / 11.0f;
    q = q * s2 + 1.0f / 9.0f;
    q = q * s2 + 1.0f / 7.0f;
    q = q * s2 + 1.0f / 5.0f;
    q = q * s2 + 1.0f / 3.0f;
    q = q * s2 + 1.0f;
    return (float)e * OG_LN2 + (s + s) * q;
}

static float og_sin_poly(float a) {  /* a in [0, pi/4] */
    float a2 = a * a;
    float p = 1.0f / 362880.0f;
    p = p * a2 - 1.0f / 5040.0f;
    p = p * a2 + 1.0f / 120.0f;
    p = p * a2 - 1.0f / 6.0f;
    p = p * a2 + 1.0f;
    return p * a;
}
static float og_cos_poly(float a) {
    float a2 = a * a;
    float p = -1.0f / 3628800.0f;
    p = p * a2 + 1.0f / 40320.0f;
    p = p * a2 - 1.0f / 720.0f;
    p = p * a2 + 1.0f / 24.0f;
    p = p * a2 - 0.5f;
    p = p * a2 + 1.0f;
    return p;
}

/* sin and cos of 2 pi t, t in [0, 1) */
void og_sincos2pi(float t, float *s, float *c) {
    float t4 = t * 4.0f;
    float kf = floorf(t4);
    int k = (int)kf;
    float f = t4 - kf; /* exact */
    float sa, ca;
    const float HALF_PI = 1.57079632679489662f;
    if (f <= 0.5f) {
        float a = f * HALF_PI;
        sa = og_sin_poly(a); ca = og_cos_poly(a);
    } else {
        float a = (1.0f - f) * HALF_PI;
        sa = og_cos_poly(a); ca = og_sin_poly(a);
    }
    switch (k & 3) {
        case 0: *s = sa; *c = ca; break;
        case 1: *s = ca; *c = -sa; break;
        case 2: *s = -sa; *c = -ca; break;
        default: *s = -ca; *c = sa; break;
    }
}

static float og_uniform(uint32_t x) { return (float)(2u * (x >> 9) + 1u) * 0x1p-24f; }

/* the four normals of VN quad q of sample s */
void og_normals4(uint64_t job, uint64_t s, uint32_t q, float g[4]) {
    uint32_t c[4] = {q, (uint32_t)s, (uint32_t)(s >> 32), 0u};
    og_philox(c, (uint32_t)job, (uint32_t)(job >> 32));
    for (int pr = 0; pr < 2; pr++) {
        float ua = og_uniform(c[2 * pr]), ub = og_uniform(c[2 * pr + 1]);
        float r = sqrtf(-2.0f * og_logf(ua));
        float sn, cs;
        og_sincos2pi(ub, &sn, &cs);
        g[2 * pr] = r * cs;
        g[2 * pr + 1] = r * sn;
    }
}

typedef struct {
    double ebn0_db, rate, mu;
    uint64_t job;
    int K, sat, alpha_num, alpha_shift;
} og_is_params;

/* sigma^2, the float constants and the log-weight coefficients */
static void og_is_consts(const og_is_params *p, float *sigf, float *muf, float *cq, double *A, double *Bc) {
    double ebn0 = pow(10.0, p->ebn0_db / 10.0);
    double s2 = 1.0 / (2.0 * p->rate * ebn0);
    *sigf = (float)sqrt(s2);
    *muf = (float)p->mu;
    *cq = (float)(16.0 / s2);
    *A = p->mu / s2;
    *Bc = p->mu * p->mu / (2.0 * s2);
}

/* The channel quantizer: 8 * (2 y / sigma^2) = y * cq with cq = 16 / sigma^2
 * in single precision, rounded half away from zero (roundf), saturated to
 * [-sat, sat]. */
int og_is_quant(float y, float cq, int sat) {
    float lq = roundf(y * cq);
    return lq > (float)sat ? sat : lq < -(float)sat ? -sat : (int)lq;
}

/* The channel of sample s: fixed-point LLRs L[v] and the drawn noise n[v]
 * (before the shift toward T) of every variable node; inT marks T. */
static void og_is_channel_mask(const og_graph *g, const unsigned char *inT, const og_is_params *p, uint64_t s,
                               int *L, float *nv) {
    float sigf, muf, cq;
    double A, Bc;
    og_is_consts(p, &sigf, &muf, &cq, &A, &Bc);
    for (int q = 0; 4 * q < g->n; q++) {
        float gq[4];
        og_normals4(p->job, s, (uint32_t)q, gq);
        for (int j = 0; j < 4 && 4 * q + j < g->n; j++) {
            int v = 4 * q + j;
            float n = sigf * gq[j];
            float y = 1.0f + n;
            if (inT[v]) y = y - muf;
            L[v] = og_is_quant(y, cq, p->sat);
            nv[v] = n;
        }
    }
}

void og_is_channel(const og_graph *g, const int *T, int a, const og_is_params *p, uint64_t s, int *L, float *nv) {
    unsigned char *inT = (unsigned char *)calloc(g->n, 1);
    for (int t = 0; t < a; t++) inT[T[t]] = 1;
    og_is_channel_mask(g, inT, p, s, L, nv);
    free(inT);
}

/* Samples [s0, s0 + ns): fail flags and log-weights. */
void og_is_samples(const og_graph *g, const int *T, int a, const og_is_params *p, uint64_t s0, int ns,
                   unsigned char *fail, double *logw) {
    float sigf, muf, cq;
    double A, Bc;
    og_is_consts(p, &sigf, &muf, &cq, &A, &Bc);
    int *L = (int *)malloc(sizeof(int) * g->n);
    unsigned char *inT = (unsigned char *)calloc(g->n, 1), *xb = (unsigned char *)malloc(g->n);
    float *nv = (float *)malloc(sizeof(float) * g->n);
    for (int t = 0; t < a; t++) inT[T[t]] = 1;
    for (int i = 0; i < ns; i++) {
        uint64_t s = s0 + (uint64_t)i;
        og_is_channel_mask(g, inT, p, s, L, nv);
        int kl;
        fail[i] = (unsigned char)og_decode_nms(g, L, p->K, p->sat, p->alpha_num, p->alpha_shift, 1, xb, &kl,
                                              NULL, NULL, NULL);
        double lw = 0.0;
        for (int v = 0; v < g->n; v++)
            if (inT[v]) lw = lw + ((double)nv[v] * A - Bc);
        logw[i] = lw;
    }
    free(L); free(inT); free(xb); free(nv);
}

/* ------------------------------------------------------------------ */
/* Frame-error simulation with the layered decoder (Fig. 2 setup)      */
/* ------------------------------------------------------------------ */
/* Frames f0 .. f0 + nf - 1: BPSK of the all-zero word over AWGN with
 * sigma^2 = 1 / (2 R Eb/N0), the noise of frame f the importance-sampling
 * generator's with key job and sample f (no shift); channel value
 * round-half-away(y * cq) with cq = 2 llr_scale / sigma^2 (single
 * precision), saturated to the LLR width; decoded by og_decode_lnms.  Per
 * frame: fail (x != 0), iterations, Hamming weight of x. */
void og_lnms_frames(const og_graph *g, double ebn0_db, double rate, double llr_scale, uint64_t job, uint64_t f0,
                    int nf, int K, int llr_bits, int c2v_bits, int v2c_bits, int an, int as, unsigned char *fail,
                    int *iters, int *weight) {
    double s2 = 1.0 / (2.0 * rate * pow(10.0, ebn0_db / 10.0));
    float sigf = (float)sqrt(s2), cq = (float)(2.0 * llr_scale / s2);
    int lim = (1 << (llr_bits - 1)) - 1;
    int *L = (int *)malloc(sizeof(int) * g->n);
    unsigned char *x = (unsigned char *)malloc(g->n);
    for (int i = 0; i < nf; i++) {
        for (int q = 0; 4 * q < g->n; q++) {
            float gq[4];
            og_normals4(job, f0 + (uint64_t)i, (uint32_t)q, gq);
            for (int j = 0; j < 4 && 4 * q + j < g->n; j++) {
                float y = 1.0f + sigf * gq[j];
                L[4 * q + j] = og_is_quant(y, cq, lim);
            }
        }
        int kl;
        fail[i] = (unsigned char)og_decode_lnms(g, L, K, llr_bits, c2v_bits, v2c_bits, an, as, x, &kl);
        iters[i] = kl;
        int w = 0;
        for (int v = 0; v < g->n; v++) w += x[v];
        weight[i] = w;
    }
    free(L);
    free(x);
}
