"""Oracle pins: the decoders, the impulse/bisection loop and the whole
enumeration on the tiny code.

The paper leaves the enumeration decoder open, so the min-sum arithmetic is
pinned by hand-computed iterations, the sum-product by exact MAP on a
cycle-free code (belief propagation is exact on trees), and the enumeration
by invariants the method must satisfy (the (a,b) recount, cycle-closure,
codewords at b = 0, circulant-shift equivariance) and by brute force.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _csr(n, rows):
    rp = np.cumsum([0] + [len(r) for r in rows])
    ci = np.concatenate([np.sort(np.array(r, dtype=np.int32)) for r in rows])
    return synth.csr_code(n, len(rows), rp, ci)


def toy6():
    # checks c0 = {0,1,2}, c1 = {2,3,4}, c2 = {0,4,5}: one 6-cycle 0-2-4
    return _csr(6, [[0, 1, 2], [2, 3, 4], [0, 4, 5]])


def test_nms_hand_trace():
    g = oracle.Graph(toy6())
    L = np.array([16, 16, -40, 16, 16, 16])
    # iteration 1 (q = L):
    #  c0 -> 0: others {16,-40}: -(3*16>>2) = -12;  -> 1: -12;  -> 2: +12
    #  c1 -> 2: +12;  -> 3: -12;  -> 4: -12;   c2 -> 0,4,5: +12
    #  P = [16-12+12, 16-12, -40+12+12, 16-12, 16-12+12, 16+12]
    f, xb, kl, u = g.decode_nms(L, K=1)
    assert kl == 1 and list(u) == [2, 2] and f
    assert g.last_P.tolist() == [16, 4, -16, 4, 16, 28]
    # iteration 2: q(v->c) = P - r: c0 gets [28, 16, -28], c1 [-28, 16, 28], c2 [4, 4, 16]
    #  c0 -> 0: -12, -> 1: -(3*28>>2) = -21, -> 2: +12;  c1 -> 2: +12, -> 3: -21, -> 4: -12
    #  c2 -> 0: +(3*4>>2) = +3, -> 4: +3, -> 5: +3
    #  P = [16-12+3, 16-21, -40+12+12, 16-21, 16-12+3, 16+3]; x = {1,2,3}, a codeword
    f, xb, kl, u = g.decode_nms(L, K=20)
    assert kl == 2 and list(u) == [2, 2, 0] and f
    assert g.last_P.tolist() == [7, -5, -16, -5, 7, 19]
    # girth 6: window starts at 3 > K_last, so x* = x_{K_last}
    assert np.flatnonzero(xb).tolist() == [1, 2, 3]


def test_nms_alpha_floor_then_sign():
    g = oracle.Graph(toy6())
    L = np.array([15, 13, -40, 15, 15, 15])
    # c0 -> 0: -(3*13>>2) = -9, -> 1: -(3*15>>2) = -11 (not floor(-11.25)), -> 2: +9
    # c1 -> 2: +11, -> 3: -11, -> 4: -11; c2 -> 0,4,5: +11
    g.decode_nms(L, K=1)
    assert g.last_P.tolist() == [15 - 9 + 11, 13 - 11, -40 + 9 + 11, 15 - 11, 15 - 11 + 11, 15 + 11]


def test_nms_saturation():
    g = oracle.Graph(toy6())
    # with sat = 20: q(2->c) = clamp(-16 - 12) = -20 instead of -28, so c0 -> 1
    # gets -(3*min(28,20)>>2) = -15 in iteration 2
    L = np.array([16, 16, -20, 16, 16, 16])
    g.decode_nms(L, K=1, sat=20)
    P1 = g.last_P.tolist()
    assert P1 == [16, 4, 4, 4, 16, 28]


def test_success_at_iteration_zero_when_amplitude_below_base():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    cands = g.candidates(3, 0)
    rng = np.random.default_rng(0)
    for ci in rng.choice(len(cands), 20, replace=False):
        I = cands[ci, 1:1 + cands[ci, 0]]
        for A in (0, 7, 16):
            L = np.full(g.n, 16)
            L[I] = 16 - A
            f, xb, kl, u = g.decode_nms(L, K=20)
            assert not f and kl == 0 and u.tolist() == [0]


def tree_code():
    # cycle-free: c0 = {0,1,2}, c1 = {2,3,4}, c2 = {4,5,6}, c3 = {1,7}
    return _csr(8, [[0, 1, 2], [2, 3, 4], [4, 5, 6], [1, 7]])


def test_spa_equals_map_on_tree():
    g = oracle.Graph(tree_code())
    H = g.dense().astype(np.int64)
    rng = np.random.default_rng(3)
    cws = [np.array(x) for x in itertools.product([0, 1], repeat=8)
           if not ((H @ np.array(x)) % 2).any()]
    for _ in range(5):
        L = rng.normal(1.0, 1.5, 8).astype(np.float32)
        P = g.spa_posterior(L, K=10)
        # exact bitwise MAP LLR: log sum_{x: x_v=0} e^{-L.x} - log sum_{x: x_v=1} e^{-L.x}
        w = np.array([np.exp(-(L.astype(np.float64) * x).sum()) for x in cws])
        X = np.array(cws)
        for v in range(8):
            want = np.log(w[X[:, v] == 0].sum()) - np.log(w[X[:, v] == 1].sum())
            assert abs(P[v] - want) < 2e-4, (v, P[v], want)


def test_spa_decode_trivial_and_codeword():
    g = oracle.Graph(toy6())
    f, xb, kl, u = g.decode_spa(np.full(6, 2.0, np.float32), K=10)
    assert not f and kl == 0
    L = np.full(6, 2.0, np.float32)
    L[[1, 2, 3]] = -5.0  # {1,2,3} is a codeword: stops at once, failed
    f, xb, kl, u = g.decode_spa(L, K=10)
    assert f and kl == 0 and np.flatnonzero(xb).tolist() == [1, 2, 3]


@pytest.fixture(scope="module")
def qc96_enum():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    res = g.enumerate(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"],
                      max_size=w["max_size"], cycle_len=w["cycle_len"])
    return w, g, res


def test_bisection_against_linear_scan(qc96_enum):
    w, g, res = qc96_enum
    rng = np.random.default_rng(11)
    mono = 0
    picks = rng.choice(len(res.cands), 12, replace=False)
    for ci in picks:
        I = res.cands[ci, 1:1 + res.cands[ci, 0]]
        fails = []
        for A in range(0, 1024):
            L = np.full(g.n, 16)
            L[I] = max(-511, 16 - A)
            fails.append(g.decode_nms(L, K=20)[0])
        fails = np.array(fails)
        thr = res.thr[ci]
        if not fails[1023]:
            assert thr == -1
            continue
        assert fails[thr] and thr >= 17
        first = int(np.argmax(fails))
        if fails[first:].all():
            mono += 1
            assert thr == first
    assert mono >= 1


def test_shift_equivariance(qc96_enum):
    w, g, res = qc96_enum
    Z = g.Z
    rng = np.random.default_rng(2)
    for ci in rng.choice(len(res.cands), 25, replace=False):
        I = res.cands[ci, 1:1 + res.cands[ci, 0]]
        s = int(rng.integers(1, Z))
        Is = (I // Z) * Z + (I % Z + s) % Z
        for A in (40, 200, 1023):
            L = np.full(g.n, 16)
            L[I] = max(-511, 16 - A)
            Ls = np.full(g.n, 16)
            Ls[Is] = max(-511, 16 - A)
            f1, x1, k1, u1 = g.decode_nms(L, K=20)
            f2, x2, k2, u2 = g.decode_nms(Ls, K=20)
            assert f1 == f2 and k1 == k2 and np.array_equal(u1, u2)
            v1 = np.flatnonzero(x1)
            assert sorted(((v1 // Z) * Z + (v1 % Z + s) % Z).tolist()) == np.flatnonzero(x2).tolist()
        r2 = g.enumerate(np.array([[len(Is)] + sorted(Is.tolist()) + [-1] * (4 - len(Is))], np.int32),
                         K=20, base_llr=16, amp_steps=10)
        assert r2.thr[0] == res.thr[ci]
        if res.ts[ci] >= 0:
            assert r2.ts_list[0].key == res.ts_list[res.ts[ci]].key


def test_enumeration_invariants(qc96_enum):
    w, g, res = qc96_enum
    H = g.dense().astype(np.int64)
    Z = g.Z
    assert len(res.cands) == len(set(map(tuple, res.cands.tolist())))
    seen = set()
    for t in res.ts_list:
        T = list(t.key)
        cnt = H[:, T].sum(axis=1)
        # (a,b) straight from the odd-degree checks of the induced subgraph
        assert (t.a, t.b) == (len(T), int((cnt % 2).sum()))
        assert t.elementary == bool((cnt <= 2).all())
        # cycle-closed: every VN keeps >= 2 checks of degree >= 2
        live = cnt >= 2
        assert all(int(live[H[:, v] > 0].sum()) >= 2 for v in T)
        # key is the brute-force minimum over all Z shifts, orbit = Z / |stab|
        best, stab = None, 0
        for s in range(Z):
            tup = tuple(sorted((v // Z) * Z + (v % Z + s) % Z for v in T))
            best = tup if best is None or tup < best else best
            stab += tup == tuple(T)
        assert t.key == best and t.orbit == Z // stab
        if t.b == 0:  # TS(a,0) is a codeword (Sec. II)
            assert not cnt.any() or not (cnt % 2).any()
        assert t.key not in seen
        seen.add(t.key)
    # counts and min thresholds agree with the per-candidate records
    for i, t in enumerate(res.ts_list):
        mask = res.ts == i
        assert t.count == int(mask.sum())
        assert t.thr == int(res.thr[mask].min())
    assert ((res.ts >= 0) <= (res.thr >= 0)).all()
    assert ((res.which == 0) == (res.ts < 0)).all()


def test_candidates_brute_force_definition():
    # every set of <= 3 VNs containing some u with the others within Tanner
    # distance 4 of u, one per circulant orbit
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense().astype(np.int64)
    A = (H.T @ H > 0).astype(np.int64)
    np.fill_diagonal(A, 0)
    near = (A > 0) | (A @ A > 0)
    np.fill_diagonal(near, False)
    Z = g.Z
    keys = set()
    n = g.n
    for S in itertools.chain(((v,) for v in range(n)), itertools.combinations(range(n), 2),
                             itertools.combinations(range(n), 3)):
        if any(all(near[u, t] for t in S if t != u) for u in S):
            best = min(tuple(sorted((v // Z) * Z + (v % Z + s) % Z for v in S)) for s in range(Z))
            keys.add(best)
    got = set(tuple(int(x) for x in r[1:1 + r[0]]) for r in g.candidates(3, 0))
    assert got == keys
    assert len(got) == 9118


def test_series_tanh_atanh_error_bounds():
    # the decoder's tanh/atanh against double-precision math: a few ulp
    xs = np.concatenate([np.linspace(-15, 15, 4001), np.geomspace(1e-8, 1, 400), -np.geomspace(1e-8, 1, 400)])
    for x in xs.astype(np.float32):
        got, want = oracle.tanhf(x), np.tanh(np.float64(x))
        assert abs(got - want) <= 4 * np.spacing(np.float32(abs(want)) if want else np.float32(1e-45)) + 1e-45, x
    ps = np.concatenate([np.linspace(-0.999, 0.999, 4001), np.geomspace(1e-8, 0.9999, 400),
                         -np.geomspace(1e-8, 0.9999, 400), [0.9999999, -0.9999999]]).astype(np.float32)
    for p in ps:
        got, want = oracle.atanhf(p), np.arctanh(np.float64(p))
        assert abs(got - want) <= 4 * np.spacing(np.float32(abs(want))) + 1e-45, p
    assert oracle.tanhf(0.0) == 0.0 and oracle.atanhf(0.0) == 0.0
    assert oracle.tanhf(20.0) == 1.0


def _xstar_cases(code, K, n_trials, seed):
    """Decodes of noisy channel values with the x_k trace; u_k recomputed from
    H independently of the decoder."""
    g = oracle.Graph(code)
    H = g.dense().astype(np.int64)
    ws = max(1, g.girth() // 2)
    rng = np.random.default_rng(seed)
    for _ in range(n_trials):
        L = np.round(rng.normal(16, 14, g.n)).astype(np.int32)
        f, xb, kl, u = g.decode_nms(L, K=K, trace=True)
        xt = g.last_trace
        assert np.array_equal((H @ xt.T.astype(np.int64) % 2).sum(0), u)
        yield ws, kl, u, xt, xb


@pytest.mark.parametrize("name", ["qc96", "qc2640"])
def test_best_pattern_first_minimum_in_window(name):
    # Sec. III: the potential trapping set is S(min_iter w_H(H x_iter)) with the
    # list starting at x_floor(girth/2).  Reading: x* = x_k at the FIRST k in
    # [max(1, floor(g/2)), K_last] with minimal u_k; x_{K_last} when K_last is
    # below the window.  Each case below is one that a wrong rule gets wrong:
    # taking the last minimum (a tie with differing patterns), a window that
    # starts one late (the unique minimum sits at floor(g/2)) or one early (a
    # smaller u_k just before the window).
    w = synth.workload(name)
    seen = {"tie": 0, "at_start": 0, "before_start": 0, "short": 0}
    for ws, kl, u, xt, xb in _xstar_cases(w["code"], 20 if name == "qc96" else 30, 3000 if name == "qc96" else 150,
                                          seed=5):
        if kl < ws:
            assert np.array_equal(xb, xt[kl])
            seen["short"] += 1
            continue
        win = u[ws:kl + 1]
        ks = [ws + i for i in np.flatnonzero(win == win.min())]
        assert np.array_equal(xb, xt[ks[0]])
        if len(ks) >= 2 and not np.array_equal(xt[ks[0]], xt[ks[-1]]):
            seen["tie"] += 1
        if ks == [ws] and kl > ws:
            late = ws + 1 + int(np.argmin(u[ws + 1:kl + 1]))
            if not np.array_equal(xt[ws], xt[late]):
                seen["at_start"] += 1
        if ws >= 2 and u[ws - 1] < win.min() and not np.array_equal(xt[ws - 1], xt[ks[0]]):
            seen["before_start"] += 1
    if name == "qc96":
        assert all(c > 0 for c in seen.values()), seen
    else:
        assert seen["tie"] > 0, seen
