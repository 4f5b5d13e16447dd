"""Oracle pins: cycles as closed exponent chains (Prop. 1), their EMD
(Sec. II, Table II) and the per-node cycle densities (Table V) behind the
iteration budgets.

Pinned to the paper's Table II (Code 1, cycle lengths 4 to 10), to the
non-backtracking matrix (the number of closed walks that never step straight
back is the trace of a power of Hashimoto's edge matrix), to a brute-force
class count written separately here, and to the simple-cycle counts of the
test helpers."""
import multiprocessing as mp
from collections import Counter

import numpy as np
import pytest

import helpers
import oracle
import synth


def _code1():
    E, Z, extra = helpers.load_code1()
    return synth.qc_code(E, Z), extra


def _walks_job(args):
    code, v, lmax = args
    return oracle.Graph(code).cycle_walks(v, lmax, emd=True)


def _spectrum(code, lmax, starts):
    with mp.get_context("spawn").Pool(min(8, len(starts))) as pool:
        parts = pool.map(_walks_job, [(code, v, lmax) for v in starts])
    walks = sum(p[0] for p in parts)
    hist = sum(p[1] for p in parts)
    return walks, hist


@pytest.fixture(scope="module")
def code1_spectrum():
    code, _ = _code1()
    return _spectrum(code, 5, [j * code.Z for j in range(20)])


def test_code1_table2_rows_4_to_10(code1_spectrum):
    # Table II (Code 1): per circulant orbit, by (cycle length, EMD); the table
    # prints integers (an orbit of half size counts 1/2: 5380.5 prints 5381)
    walks, hist = code1_spectrum
    want = helpers.load_table2_code1()
    for (clen, e), count in want.items():
        l = clen // 2
        if l > 5:
            continue
        got = hist[l, e] / (2 * l)
        assert abs(got - count) <= 0.5, (clen, e, got, count)
        assert round(got + 1e-9) == count or got == count - 0.5, (clen, e, got, count)
    # no other (length, EMD) has cycles
    for l in range(2, 6):
        for e in np.flatnonzero(hist[l]):
            assert (2 * l, int(e)) in want, (2 * l, e)
    # the one half-size orbit class of 8-cycles: 5380.5
    assert hist[4, 8] / 8 == 5380.5


def _nonbacktracking_traces(g, kmax):
    # Hashimoto's matrix on directed edges of the Tanner graph:
    # B[(a->b), (b->c)] = 1 for c != a; trace(B^k) = closed walks of length k
    # that never step straight back (including at the closing step), counted
    # once per starting directed edge
    edges = []
    for c in range(g.m):
        for v in g.check_vns(c):
            edges.append((("v", v), ("c", c)))
            edges.append((("c", c), ("v", v)))
    idx = {e: i for i, e in enumerate(edges)}
    out_of = {}
    for a, b in edges:
        out_of.setdefault(a, []).append(b)
    N = len(edges)
    B = np.zeros((N, N), dtype=np.int64)
    for (a, b), i in idx.items():
        for c in out_of[b]:
            if c != a:
                B[i, idx[(b, c)]] = 1
    tr, P = [], np.eye(N, dtype=np.int64)
    for k in range(1, kmax + 1):
        P = P @ B
        tr.append(int(np.trace(P)))
    return tr


def test_closed_walks_against_hashimoto_matrix():
    # qc96: half the trace counts the walks that start at a variable node;
    # by the circulant symmetry that is Z times the walks from (j,0)
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    lmax = 6
    walks = np.zeros(lmax + 1, dtype=np.int64)
    for j in range(6):
        walks += g.cycle_walks(j * 16, lmax)
    tr = _nonbacktracking_traces(g, 2 * lmax)
    for l in range(2, lmax + 1):
        assert tr[2 * l - 1] // 2 == 16 * walks[l], l
        assert tr[2 * l - 1] % 2 == 0
    # odd lengths are impossible in a bipartite graph
    assert all(tr[k] == 0 for k in range(0, 2 * lmax, 2))


def test_class_weights_against_brute_force_classes():
    # every closed walk from every variable node of qc96, reduced to a class
    # (smallest rotation / reversal of its node sequence), counted per EMD;
    # divided by Z it must equal the oracle's weighted counts from (j,0)
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense()
    vn, cn = helpers.adjacency(H)
    Z, lmax = 16, 5

    def classes_from(v0, l):
        out = set()

        def rec(vs, cs):
            v = vs[-1]
            for c in vn[v]:
                if cs and c == cs[-1]:
                    continue
                if len(vs) == l:
                    if v != v0 and c != cs[0] and v0 in cn[c]:
                        seq = list(zip(vs, cs + [c]))
                        out.add(_canon(seq))
                    continue
                for u in cn[c]:
                    if u != v:
                        rec(vs + [u], cs + [c])

        rec([v0], [])
        return out

    hist_or = np.zeros((lmax + 1, 128), dtype=np.int64)
    for j in range(6):
        hist_or += g.cycle_walks(j * Z, lmax, emd=True)[1]
    for l in range(2, lmax + 1):
        allc = set()
        for v in range(g.n):
            allc |= classes_from(v, l)
        cnt = Counter(helpers.emd(None, H, {x for x, _ in cls}) for cls in allc)
        for e in set(cnt) | set(np.flatnonzero(hist_or[l]).tolist()):
            assert cnt[e] * 2 * l == hist_or[l, e] * Z, (l, e, cnt[e], hist_or[l, e])


def _canon(seq):
    # seq: [(v_t, c_{t+1})] of a closed walk; the class under rotation and reversal
    L = len(seq)
    vs = [s[0] for s in seq]
    cs = [s[1] for s in seq]  # cs[t] joins v_t and v_{t+1}
    forms = []
    for s in range(L):
        forms.append(tuple((vs[(s + t) % L], cs[(s + t) % L]) for t in range(L)))
        # reverse: v_s, then the check before it, v_{s-1}, ...
        forms.append(tuple((vs[(s - t) % L], cs[(s - t - 1) % L]) for t in range(L)))
    return min(forms)


@pytest.mark.parametrize("name", ["qc96", "peg1008"])
def test_node_cycle_counts_against_simple_cycles(name):
    # up to length 6 every closed walk is a simple cycle: walks / 2 = cycles through v
    w = synth.workload(name)
    g = oracle.Graph(w["code"])
    H = g.dense()
    vn, cn = helpers.adjacency(H)
    for v in (0, 5, 17, 95):
        walks = g.cycle_walks(v, 3)
        assert walks[2] == 2 * len(helpers.cycles_through_vn(vn, cn, v, 2))
        assert walks[3] == 2 * len(helpers.cycles_through_vn(vn, cn, v, 3))


def test_code1_table5_column_densities_from_walks():
    # Table V: 6-cycles through a column block per node, (cycles through (j,0)) / 3
    code, extra = _code1()
    g = oracle.Graph(code)
    from test_oracle_graph import _printed_matches
    for j in range(20):
        walks = g.cycle_walks(j * code.Z, 3)
        assert _printed_matches(walks[3] / 2 / 3, extra["col_cyc6"][j]), j
        assert _printed_matches(walks[2] / 2 / 2, extra["col_cyc4"][j]), j


def _cycle_weights(code):
    g = oracle.Graph(code)
    vn, cn = helpers.adjacency(g.dense())
    return np.array([2 * len(helpers.cycles_through_vn(vn, cn, v, 2)) + len(helpers.cycles_through_vn(vn, cn, v, 3))
                     for v in range(g.n)])


def test_iteration_budget_per_candidate():
    # Sec. III: the iteration count follows the density of cycles through the
    # impulse nodes; reading: K(I) = kmin + ceil((K - kmin) wref / (wref + W(I))),
    # W(I) = sum over I of 2 c4(v) + c6(v).  Each candidate must give exactly
    # what a plain run with K = K(I) gives.
    code = helpers_code_with_4_cycles()
    g = oracle.Graph(code)
    W = _cycle_weights(code)
    assert W.max() > W.min()
    K, kmin, wref = 20, 4, 6
    p = dict(base_llr=16, amp_steps=10, max_size=2)
    cands = g.candidates(2, 0)
    res = g.enumerate(cands, K=K, budget_wref=wref, budget_kmin=kmin, **p)
    budgets = set()
    for i, row in enumerate(cands):
        I = row[1:1 + row[0]]
        Wi = int(W[I].sum())
        Kc = kmin + -(-(K - kmin) * wref // (wref + Wi))
        budgets.add(Kc)
        one = g.enumerate(row[None], K=Kc, **p)
        assert (res.thr[i], res.decodes[i], res.iters[i]) == (one.thr[0], one.decodes[0], one.iters[0]), row
    assert len(budgets) > 2


def helpers_code_with_4_cycles():
    # a 3 x 6 QC base with one repeated shift difference (4-cycles through some columns)
    return synth.qc_code([[0, 1, 2, 3, 4, 5], [0, 2, 4, 6, 8, 10], [0, 3, 6, 1, 12, 15]], 16)


def test_converged_decode_statistics():
    # the two-stage schedule starts the lists at ceil(average iterations of the
    # decodes that converged to the all-zero word); recount those decodes by
    # running the bisection with the oracle's decoder
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    cands = g.candidates(2, 0)[::40]
    res = g.enumerate(cands, K=20, base_llr=16, amp_steps=10, max_size=2)
    ok = okit = 0
    for row in cands:
        I = row[1:1 + row[0]]
        lo, hi = 0, 1023

        def dec(A):
            L = np.full(g.n, 16)
            L[I] = max(-511, 16 - A)
            f, _, kl, _ = g.decode_nms(L, K=20)
            return f, kl

        f, kl = dec(hi)
        runs = [(f, kl)]
        if f:
            for _ in range(10):
                if hi - lo <= 1:
                    break
                mid = (lo + hi) // 2
                f, kl = dec(mid)
                runs.append((f, kl))
                if f:
                    hi = mid
                else:
                    lo = mid
        ok += sum(1 for f, _ in runs if not f)
        okit += sum(kl for f, kl in runs if not f)
    assert (res.converged, res.converged_iterations) == (ok, okit)
    two = g.enumerate(cands, K=20, base_llr=16, amp_steps=10, max_size=2, list_mode=True, kstart=-1)
    ks = max(1, -(-okit // ok))
    assert two.kstart == ks
    one = g.enumerate(cands, K=20, base_llr=16, amp_steps=10, max_size=2, list_mode=True, kstart=ks)
    assert [(t.key, t.count, t.kind, t.thr) for t in two.ts_list] == [(t.key, t.count, t.kind, t.thr)
                                                                      for t in one.ts_list]
