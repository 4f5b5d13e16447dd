"""Oracle pins: Tree()/TS() sieving, (a,b) classification, canonical key and
orbit size (Sec. II-III), pinned to Table III, hand-drawn subgraphs (the
shapes of Fig. 1) and brute force."""
import itertools

import numpy as np
import pytest

import helpers
import oracle
import synth


def _csr(n, rows):
    rp = np.cumsum([0] + [len(r) for r in rows])
    ci = np.concatenate([np.sort(np.array(r, dtype=np.int32)) for r in rows])
    return synth.csr_code(n, len(rows), rp, ci)


# --- Fig. 1 shapes ------------------------------------------------------------

def ts44_code():
    # TS(4,4): one 8-cycle 0-1-2-3-0 through degree-2 checks c0..c3, each VN
    # has one more check c4..c7 reaching the rest of the graph (VNs 4..7)
    rows = [[0, 1], [1, 2], [2, 3], [3, 0], [0, 4], [1, 5], [2, 6], [3, 7],
            [4, 5], [6, 7], [4, 6], [5, 7]]
    return _csr(8, rows)


def ts53_code():
    # TS(5,3): K_{2,3} VN graph (three overlapping 8-cycles): A=0, B=1 joined
    # to x=2, y=3, z=4 by degree-2 checks; x, y, z each have one odd check
    rows = [[0, 2], [0, 3], [0, 4], [1, 2], [1, 3], [1, 4], [2, 5], [3, 6], [4, 7],
            [5, 6, 7]]
    return _csr(8, rows)


def test_fig1_ts44():
    g = oracle.Graph(ts44_code())
    T = {0, 1, 2, 3}
    assert g.tree(T) == T
    assert g.classify(T) == (4, 4, True)


def test_fig1_ts53():
    g = oracle.Graph(ts53_code())
    T = {0, 1, 2, 3, 4}
    assert g.tree(T) == T
    assert g.classify(T) == (5, 3, True)


def test_tree_drops_pendants_and_paths():
    g = oracle.Graph(ts44_code())
    assert g.tree({0, 1, 2, 3, 4}) == {0, 1, 2, 3}   # 4 hangs on one check
    assert g.tree({0, 1, 2}) == set()                # a path has no cycle
    assert g.tree({4, 5, 6, 7}) == {4, 5, 6, 7}       # the other 8-cycle


def test_ts_closure_and_s2():
    # X = path 0-1-2 of the 8-cycle: Tree(X) is empty, TS(X) adds 3 (two
    # checks in N(X)), and Tree(TS(X)) is the cycle: the S2 sieve of Sec. III
    g = oracle.Graph(ts44_code())
    assert g.ts_closure({0, 1, 2}) == {0, 1, 2, 3}
    x = np.zeros(8, np.uint8)
    x[[0, 1, 2]] = 1
    which, T = g.extract(x, [])
    assert which == 2 and T == {0, 1, 2, 3}
    x[:] = 0
    x[[0, 1, 2, 3, 4]] = 1
    which, T = g.extract(x, [])
    assert which == 1 and T == {0, 1, 2, 3}
    x[:] = 0
    which, T = g.extract(x, [0])  # a lone VN: no cycle even after closure
    assert which == 0 and T == set()
    # {0, 5}: 1 and 4 each see two checks of N(X) and close the 8-cycle 0-1-5-4
    assert g.ts_closure({0, 5}) == {0, 1, 4, 5}
    which, T = g.extract(x, [0, 5])
    assert which == 2 and T == {0, 1, 4, 5}


def test_ab_independent_recount_random_sets():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense().astype(np.int64)
    rng = np.random.default_rng(5)
    for _ in range(200):
        k = int(rng.integers(1, 12))
        T = set(rng.choice(g.n, k, replace=False).tolist())
        cnt = H[:, sorted(T)].sum(axis=1)
        assert g.classify(T) == (k, int((cnt % 2).sum()), bool((cnt <= 2).all()))
        # Tree(T) is a fixed point with every VN on >= 2 checks of degree >= 2
        Tt = g.tree(T)
        assert Tt <= T and g.tree(Tt) == Tt
        if Tt:
            c2 = H[:, sorted(Tt)].sum(axis=1) >= 2
            assert all(int(c2[H[:, v] > 0].sum()) >= 2 for v in Tt)


# --- planted codeword: TS(a,0) is a codeword (Sec. II) --------------------------

def planted_k4_code():
    # VNs 0..3 pairwise joined by the 6 checks c0..c5 (the edges of K4), so
    # {0,1,2,3} is a weight-4 codeword; each K4 check also holds one VN of
    # 4..9, which are tied together by c6..c10 (all VNs have degree 3)
    rows = [[0, 1, 4], [0, 2, 5], [0, 3, 6], [1, 2, 7], [1, 3, 8], [2, 3, 9],
            [4, 5, 6], [7, 8, 9], [4, 7], [5, 8], [6, 9]]
    return _csr(10, rows)


def test_planted_codeword_is_lightest():
    H = oracle.Graph(planted_k4_code()).dense().astype(np.int64)
    x = np.zeros(10, np.int64)
    x[:4] = 1
    assert not ((H @ x) % 2).any()
    for k in (1, 2, 3):
        for S in itertools.combinations(range(10), k):
            y = np.zeros(10, np.int64)
            y[list(S)] = 1
            assert ((H @ y) % 2).any()


def test_planted_codeword_found_as_ts_a0():
    g = oracle.Graph(planted_k4_code())
    res = g.enumerate(np.array([[4, 0, 1, 2, 3]], np.int32), K=20, base_llr=16, amp_steps=10)
    # A <= base leaves every LLR >= 0 (decodes at iteration 0); A = base + 1
    # makes the impulse a codeword: the decoder stops at once on it
    assert res.thr[0] == 17
    assert len(res.ts_list) == 1
    t = res.ts_list[0]
    assert (t.a, t.b, t.key) == (4, 0, (0, 1, 2, 3))


# --- canonical form and orbit (graph automorphism) ----------------------------

def _brute_key(T, Z):
    best = None
    stab = 0
    base = sorted(T)
    for s in range(Z):
        tup = sorted((v // Z) * Z + (v % Z + s) % Z for v in T)
        if best is None or tup < best:
            best = tup
        stab += tup == base
    return tuple(best), Z // stab


@pytest.mark.parametrize("name", ["qc96", "qc2640"])
def test_canon_matches_brute_force(name):
    w = synth.workload(name)
    g = oracle.Graph(w["code"])
    Z = g.Z
    rng = np.random.default_rng(1)
    for _ in range(100):
        k = int(rng.integers(1, 9))
        T = rng.choice(g.n, k, replace=False).tolist()
        key, orbit = g.canon(T)
        assert (key, orbit) == _brute_key(T, Z)
        s = int(rng.integers(0, Z))
        T2 = [(v // Z) * Z + (v % Z + s) % Z for v in T]
        assert g.canon(T2) == (key, orbit)


def test_orbit_with_stabilizer():
    g = oracle.Graph(synth.qc_code([[0, 1], [2, 3]], 16))
    assert g.canon([0, 8]) == ((0, 8), 8)
    assert g.canon([0, 4, 8, 12]) == ((0, 4, 8, 12), 4)
    assert g.canon([3, 19]) == ((0, 16), 16)


def test_non_qc_key_is_sorted_set():
    g = oracle.Graph(synth.workload("peg1008")["code"])
    assert g.canon([9, 3, 700]) == ((3, 9, 700), 1)


# --- Table III: TS(2,2) = TS(3,2) = 128 on Code 1 ----------------------------

def test_code1_table3_small_ts_bruteforce():
    E, Z, _ = helpers.load_code1()
    g = oracle.Graph(synth.qc_code(E, Z))
    H = g.dense().astype(np.int64)
    vn, cn = helpers.adjacency(H)
    N2 = [set(u for c in vn[v] for u in cn[c]) - {v} for v in range(g.n)]

    def closed(S):
        cnt = H[:, sorted(S)].sum(axis=1)
        live = cnt >= 2
        return all(int(live[vn[v]].sum()) >= 2 for v in S)

    found = {}
    checked_nonclosed = 0
    for j in range(20):
        v0 = j * Z
        for u in N2[v0]:
            sets = [frozenset((v0, u))]
            sets += [frozenset((v0, u, w)) for w in (N2[v0] | N2[u]) - {v0, u}]
            for S in sets:
                if closed(S):
                    assert g.tree(S) == set(S)
                    a, b, _ = g.classify(S)
                    key, orbit = g.canon(sorted(S))
                    found[key] = (a, b, orbit)
                elif checked_nonclosed < 300:
                    checked_nonclosed += 1
                    assert g.tree(S) != set(S)
    counts = {}
    for a, b, orbit in found.values():
        counts[(a, b)] = counts.get((a, b), 0) + orbit
    for (a, b), want in helpers.load_table3_code1().items():
        assert counts.get((a, b), 0) == want, (a, b, counts)
