"""Oracle pins for the ordered-list mode (Sec. III): for a failing impulse,
the sets S1(x_k) = Tree(X_k) and S2(x_k) = Tree(TS(X_k)), X_k = supp(x_k) u I,
for k = floor(girth/2) .. K_last of the decode at the threshold amplitude,
every non-empty one a trapping set.

The list is rebuilt here from the decoder's x_k trace with an independent
dense-matrix restatement of Tree() (2-core peeling) and TS() (one closure
pass) and compared with the oracle's list mode; the (a, b) of every listed set
is recounted from the dense matrix, and the single-pattern mode's sets must
be among the listed ones."""
import numpy as np

import oracle
import synth

P = dict(K=20, base_llr=16, amp_steps=10)


def _tree_dense(H, S):
    S = set(S)
    while True:
        keep_c = [c for c in range(H.shape[0]) if sum(H[c, v] for v in S) >= 2]
        deg = {v: sum(H[c, v] for c in keep_c) for v in S}
        drop = {v for v, d in deg.items() if d <= 1}
        if not drop:
            return S
        S -= drop


def _ts_dense(H, S):
    S = set(S)
    NS = {c for c in range(H.shape[0]) if any(H[c, v] for v in S)}
    add = {v for v in range(H.shape[1]) if v not in S and sum(1 for c in NS if H[c, v]) >= 2}
    return S | add


def _ab_dense(H, T):
    T = sorted(T)
    deg = H[:, T].sum(axis=1)
    return len(T), int(np.sum(deg % 2 == 1))


def _list_keys(g, H, cand, thr, wstart):
    """The candidate's ordered list at its threshold, restated from the paper."""
    nI = int(cand[0])
    I = [int(v) for v in cand[1:1 + nI]]
    L = np.full(g.n, P["base_llr"], np.int32)
    L[I] = max(P["base_llr"] - thr, -511)
    fail, _, kl, _ = g.decode_nms(L, P["K"], trace=True)
    assert fail
    keys = set()
    for k in range(wstart, kl + 1):
        X = set(np.flatnonzero(g.last_trace[k]).tolist()) | set(I)
        for T in (_tree_dense(H, X), _tree_dense(H, _ts_dense(H, X))):
            if T:
                keys.add(g.canon(sorted(T))[0])
    return keys


def test_list_mode_equals_restatement_on_sampled_candidates():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense().astype(np.int64)
    wstart = max(1, g.girth() // 2)
    cands = g.candidates(3, 0)
    rng = np.random.default_rng(8)
    sample = cands[np.sort(rng.choice(len(cands), 60, replace=False))]
    single = g.enumerate(sample, **P)
    failing = sample[single.thr >= 0]
    thr = single.thr[single.thr >= 0]
    assert len(failing) >= 10
    lst = g.enumerate(failing, list_mode=True, **P)
    want = set()
    for c, t in zip(failing, thr):
        want |= _list_keys(g, H, c, int(t), wstart)
    got = {t.key for t in lst.ts_list}
    assert got == want
    # every listed set is cycle-closed, with (a, b) recounted from the matrix
    for t in lst.ts_list:
        assert _tree_dense(H, t.key) == set(t.key)
        assert (t.a, t.b) == _ab_dense(H, t.key)
        assert t.kind in (1, 2, 3)
    # the list holds several sets per failing candidate on this code
    assert len(lst.ts_list) > len({t.key for t in g.enumerate(failing, **P).ts_list})


def test_single_pattern_sets_are_in_the_list():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    single = g.enumerate(max_size=2, **P)
    lst = g.enumerate(max_size=2, list_mode=True, **P)
    got = {t.key for t in lst.ts_list}
    missing = [t.key for t in single.ts_list if t.key not in got]
    assert not missing
    # counts: a set is counted once per candidate whose list holds it
    n_fail = int(np.sum(single.thr >= 0))
    assert all(1 <= t.count <= n_fail for t in lst.ts_list)
    # thresholds: each set keeps the smallest threshold among its candidates
    assert min(t.thr for t in lst.ts_list) == int(single.thr[single.thr >= 0].min())


def test_list_window():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    cands = g.candidates(2, 0)[:400]
    late = g.enumerate(cands, list_mode=True, kstart=P["K"] + 1, **P)
    assert late.ts_list == []  # the window starts after the last iteration
    early = {t.key for t in g.enumerate(cands, list_mode=True, kstart=1, **P).ts_list}
    default = {t.key for t in g.enumerate(cands, list_mode=True, **P).ts_list}
    assert default <= early
