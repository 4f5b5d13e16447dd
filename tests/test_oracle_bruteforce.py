"""Brute-force subgraph enumeration of all elementary, cycle-closed trapping
sets with a <= 5 on the tiny QC code, checked against what the oracle's
enumeration reports.  Coverage (the share of them the impulse method finds)
is reported, not gated: the method is a heuristic (Sec. III)."""
import numpy as np

import oracle
import synth


def _connected_sets(adj, v0, kmax, ok):
    """ESU enumeration of connected vertex sets with minimum vertex v0 and
    size <= kmax whose every prefix on the search path satisfies ok()."""
    out = []

    def ext(sub, extension, excl):
        out.append(sub)
        if len(sub) == kmax:
            return
        extension = list(extension)
        while extension:
            w = extension.pop()
            s2 = sub | {w}
            if not ok(s2):
                continue
            nb = [u for u in adj[w] if u > v0 and u not in excl]
            ext(s2, extension + nb, excl | set(adj[w]))

    ext(frozenset([v0]), [u for u in adj[v0] if u > v0], set(adj[v0]) | {v0})
    return out


def test_elementary_ts_bruteforce_a_le_5():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense().astype(np.int64)
    Z = g.Z
    vn = [np.flatnonzero(H[:, v]) for v in range(g.n)]
    adj = [sorted(set(np.flatnonzero(H[vn[v]].sum(axis=0))) - {v}) for v in range(g.n)]

    def elementary(S):
        return H[:, sorted(S)].sum(axis=1).max() <= 2

    brute = {}
    for j in range(g.n // Z):
        for S in _connected_sets(adj, j * Z, 5, elementary):
            cnt = H[:, sorted(S)].sum(axis=1)
            live = cnt == 2
            if all(int(live[vn[v]].sum()) >= 2 for v in S):
                key = min(tuple(sorted((v // Z) * Z + (v % Z + s) % Z for v in S))
                          for s in range(Z))
                brute[key] = (len(S), int((cnt % 2).sum()))
    assert brute, "the tiny code has short cycles, so small TS exist"
    res = g.enumerate(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"],
                      max_size=w["max_size"], cycle_len=w["cycle_len"])
    small = [t for t in res.ts_list if t.a <= 5 and t.elementary]
    for t in small:
        assert t.key in brute, t
        assert brute[t.key] == (t.a, t.b)
    found = sum(1 for k in brute if k in {t.key for t in small})
    print(f"\nelementary TS with a<=5: {len(brute)} exist, impulse method found {found}")
