"""GPU parity: the CUDA library (through its C ABI) against the oracle.

Fixed-point min-sum must be bit-exact: the same canonical candidates, per
candidate the same threshold amplitude, trapping set, sieve, number of
decodes and iterations, and the same list of distinct trapping sets
(a, b, key, orbit, count, min threshold, elementary flag).  The sum-product
variant must give thresholds within 1e-3 and the same trapping set wherever
the thresholds agree.  Small codes are compared in full; the full-size
workloads run in the bench's launch configuration and are compared on
sampled candidates plus invariants that hold at any size.
"""
import numpy as np
import pytest

import helpers
import oracle
import synth
from gpu_helpers import (lib_cand_tuples, lib_records, lib_ts, oracle_cand_tuples, oracle_records, oracle_ts,
                         run_lib)

pytestmark = pytest.mark.gpu

NMS = dict(K=20, base_llr=16, amp_steps=10, max_size=3, cycle_len=0)


def _params(w, **over):
    p = dict(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"], max_size=w["max_size"],
             cycle_len=w["cycle_len"])
    p.update(over)
    return p


def _full_compare(v, res):
    assert sorted(lib_cand_tuples(v)) == sorted(oracle_cand_tuples(res.cands))
    assert lib_records(v) == oracle_records(res)
    assert lib_ts(v) == oracle_ts(res)
    # list order: (a, b, key)
    order = [(int(a), int(b), k) for a, b, k in zip(v["a"], v["b"], v["keys"])]
    assert order == sorted(order)


@pytest.fixture(scope="module")
def qc96():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    res = g.enumerate(**_params(w))
    v = run_lib(w["code"], **_params(w))
    return w, g, res, v


def test_qc96_full_bit_exact(qc96):
    w, g, res, v = qc96
    assert len(v["cand_thr"]) == 9118
    _full_compare(v, res)


def test_qc96_stats(qc96):
    w, g, res, v = qc96
    s = v["stats"]
    assert s["n_cand"] == s["n_cand_total"] == len(res.cands)
    assert s["decodes"] == int(res.decodes.sum())
    assert s["iterations"] == int(res.iters.sum())
    assert s["edge_updates"] == g.E * int(res.iters.sum())
    assert s["acyclic"] == int(((res.thr >= 0) & (res.which == 0)).sum())
    assert s["n_ts"] == len(res.ts_list)
    assert v["info"]["girth"] == g.girth() == 6


def test_qc96_deterministic_and_shape_independent(qc96):
    w, g, res, v = qc96
    for over in (dict(), dict(warps_per_cta=1), dict(warps_per_cta=4, ctas_per_sm=1), dict(kernel=1),
                 dict(kernel=1, warps_per_cta=2), dict(kernel=2, warps_per_cta=2)):
        v2 = run_lib(w["code"], **_params(w, **over))
        assert lib_records(v2) == lib_records(v)
        assert lib_ts(v2) == lib_ts(v)


def test_qc96_shards(qc96):
    w, g, res, v = qc96
    N = len(v["cand_thr"])
    full = lib_records(v)
    tuples = lib_cand_tuples(v)
    for b, e in ((0, 1), (17, 4000), (4000, N), (N - 3, -1)):
        vs = run_lib(w["code"], **_params(w, cand_begin=b, cand_end=e))
        ee = N if e < 0 else e
        assert lib_cand_tuples(vs) == tuples[b:ee]
        assert all(full[t] == r for t, r in lib_records(vs).items())


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("over", [dict(max_size=1), dict(max_size=2), dict(K=0), dict(amp_steps=1),
                                  dict(K=7, base_llr=40, alpha_num=5, alpha_shift=3), dict(sat=63),
                                  dict(base_llr=2000, sat=1023)])
def test_qc96_parameter_edges(over, kernel):
    # kernel 1: one codeword per group; kernel 2: two per lane (16-bit halves)
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    p = _params(w, **over)
    res = g.enumerate(**p)
    v = run_lib(w["code"], kernel=kernel, **p)
    _full_compare(v, res)


@pytest.mark.parametrize("kernel", [1, 2])
def test_qc96_int8_storage_bit_exact(kernel):
    # int8 check-to-variable storage is the same decoder with sat <= 169
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    p = _params(w, sat=127)
    res = g.enumerate(**p)
    v = run_lib(w["code"], decoder="nms8", kernel=kernel, **p)
    _full_compare(v, res)


def test_qc96_spa_bit_exact():
    # both sides evaluate tanh/atanh by the same series with IEEE-rounded
    # operations, so the float decoder agrees bit for bit (well inside the
    # 1e-3 threshold tolerance)
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    p = _params(w, amp_steps=12)
    res = g.enumerate(decoder="spa", spa_clip=30.0, spa_amax=64.0, **p)
    v = run_lib(w["code"], decoder="spa", **p)
    lr, orr = lib_records(v), oracle_records(res)
    assert lr.keys() == orr.keys()
    for t, rec in orr.items():
        assert abs(lr[t][1] - rec[1]) <= 1e-3, (t, lr[t], rec)
    _full_compare(v, res)


def test_planted_codeword_and_tree_code():
    rows = [[0, 1, 4], [0, 2, 5], [0, 3, 6], [1, 2, 7], [1, 3, 8], [2, 3, 9],
            [4, 5, 6], [7, 8, 9], [4, 7], [5, 8], [6, 9]]
    rp = np.cumsum([0] + [len(r) for r in rows])
    k4 = synth.csr_code(10, len(rows), rp, np.concatenate(rows))
    g = oracle.Graph(k4)
    p = dict(K=20, base_llr=16, amp_steps=10, max_size=4)
    res = g.enumerate(**p)
    v = run_lib(k4, **p)
    _full_compare(v, res)
    assert (4, 0, 1) in {(a, b, o) for a, b, o, *_ in lib_ts(v).values()}
    tree = synth.csr_code(8, 4, [0, 3, 6, 9, 11], [0, 1, 2, 2, 3, 4, 4, 5, 6, 1, 7])
    g = oracle.Graph(tree)
    res = g.enumerate(**p)
    v = run_lib(tree, **p)
    assert v["info"]["girth"] == 0
    _full_compare(v, res)


def test_code1_table5_small_sets():
    # Table V's Code 1 has one 4-cycle orbit; the impulse on its two VNs
    # reports TS(2,2).  Full library run, oracle on a sample that includes it.
    E, Z, _ = helpers.load_code1()
    code = synth.qc_code(E, Z)
    w = dict(code=code, K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)
    v = run_lib(code, **_params(w))
    g = oracle.Graph(code)
    H = g.dense().astype(np.int64)
    pair = None
    for u in g.ball4(0):
        if int((H[:, 0] * H[:, u]).sum()) >= 2:
            pair = g.canon([0, int(u)])[0]
    assert pair is not None
    res = g.enumerate(np.array([[2, pair[0], pair[1], -1, -1]], np.int32), **_params(w))
    assert (res.ts_list[res.ts[0]].a, res.ts_list[res.ts[0]].b) == (2, 2)
    i = lib_cand_tuples(v).index(pair)
    assert int(v["cand_thr"][i]) == int(res.thr[0])
    k = v["keys"][int(v["cand_ts"][i])]
    assert k == res.ts_list[res.ts[0]].key and len(k) == 2
    _sampled_compare(w, v, 30, seed=13)


def test_batch_code_with_zero_blocks():
    # a 4 x 25 base with weight-3 and weight-4 columns, Z = 128
    code = synth.batch_codes([103])[0]
    w = dict(code=code, K=15, base_llr=16, amp_steps=8, max_size=2, cycle_len=0)
    v = run_lib(code, **_params(w))
    g = _sampled_compare(w, v, 80, seed=11)
    _ts_invariants(g, v, qc=True)


# ---------------------------------------------------------------------------
# full-size workloads: the bench's launch configuration, sampled comparison
# ---------------------------------------------------------------------------
def _sorted_rows(cv):
    cv = np.asarray(cv)
    order = np.lexsort(tuple(cv[:, k] for k in range(cv.shape[1] - 1, -1, -1)))
    return cv[order], order


def _sampled_compare(w, v, n_sample, seed, decoder="nms", tol=0.0):
    g = oracle.Graph(w["code"])
    oc = g.candidates(w["max_size"], w["cycle_len"])
    # same canonical candidate set (as sorted rows of (size, v0..v3))
    lib_rows = np.concatenate([(v["cand_vars"] >= 0).sum(1, keepdims=True), v["cand_vars"]], axis=1)
    ls, lorder = _sorted_rows(lib_rows)
    os_, _ = _sorted_rows(oc)
    assert ls.shape == os_.shape and np.array_equal(ls, os_)
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(oc), n_sample, replace=False))
    sample = os_[pick]
    res = g.enumerate(sample, decoder=decoder, **_params(w))
    keys = v["keys"]
    lkeys = _rowkey(ls, g.n)
    for j, row in enumerate(sample):
        li = lorder[np.searchsorted(lkeys, _rowkey(row[None], g.n)[0])]
        ts = int(v["cand_ts"][li])
        lkey = keys[ts] if ts >= 0 else None
        okey = res.ts_list[res.ts[j]].key if res.ts[j] >= 0 else None
        if decoder == "nms":
            assert int(v["cand_thr"][li]) == int(res.thr[j]), row
            assert lkey == okey, row
            assert int(v["cand_decodes"][li]) == int(res.decodes[j]), row
            assert int(v["cand_iters"][li]) == int(res.iters[j]), row
        else:
            assert abs(float(v["cand_thr_f"][li]) - float(res.thr_f[j])) <= tol, row
            if float(v["cand_thr_f"][li]) == float(res.thr_f[j]):
                assert lkey == okey, row
    return g


def _rowkey(rows, n):
    # (size, v0..v3) -> one int64, order-preserving (values + 1 lie in [0, n])
    rows = np.asarray(rows, dtype=np.int64) + 1
    assert 5 * (n + 1) ** 4 < 2 ** 62
    k = np.zeros(rows.shape[0], dtype=np.int64)
    for c in range(rows.shape[1]):
        k = k * (n + 1) + rows[:, c]
    return k


def _ts_invariants(g, v, qc):
    H = g.dense().astype(np.int64)
    Z = g.Z
    ts = v["cand_ts"]
    counts = np.bincount(ts[ts >= 0], minlength=len(v["keys"]))
    assert np.array_equal(counts, v["count"])
    for i, key in enumerate(v["keys"][:500]):
        cnt = H[:, list(key)].sum(axis=1)
        assert (int(v["a"][i]), int(v["b"][i])) == (len(key), int((cnt % 2).sum()))
        live = cnt >= 2
        assert all(int(live[H[:, x] > 0].sum()) >= 2 for x in key)
        if qc:
            best = min(tuple(sorted((x // Z) * Z + (x % Z + s) % Z for x in key)) for s in range(Z))
            assert best == key
        else:
            assert list(key) == sorted(key) and int(v["orbit"][i]) == 1
        mask = ts == i
        assert int(v["thr"][i]) == int(v["cand_thr"][mask].min())


@pytest.fixture(scope="module")
def peg1008():
    w = synth.workload("peg1008")
    v = run_lib(w["code"], **_params(w))
    return w, v


def test_peg1008_full_size_sampled(peg1008):
    w, v = peg1008
    g = _sampled_compare(w, v, 150, seed=7)
    _ts_invariants(g, v, qc=False)


def test_peg1008_spa_shard_sampled():
    w = synth.workload("peg1008")
    p = _params(w)
    v = run_lib(w["code"], decoder="spa", cand_begin=0, cand_end=4000, **p)
    g = oracle.Graph(w["code"])
    oc = g.candidates(w["max_size"], w["cycle_len"])
    lib_first = lib_cand_tuples(v)
    rng = np.random.default_rng(3)
    idx = np.sort(rng.choice(len(lib_first), 40, replace=False))
    rows = np.array([[len(lib_first[i])] + list(lib_first[i]) + [-1] * (4 - len(lib_first[i])) for i in idx],
                    dtype=np.int32)
    # every sampled candidate is in the oracle's own list
    oset = set(map(tuple, oc.tolist()))
    assert all(tuple(r) in oset for r in rows.tolist())
    res = g.enumerate(rows, decoder="spa", **p)
    keys = v["keys"]
    for j, i in enumerate(idx):
        assert abs(float(v["cand_thr_f"][i]) - float(res.thr_f[j])) <= 1e-3
        assert float(v["cand_thr_f"][i]) == float(res.thr_f[j])
        assert int(v["cand_iters"][i]) == int(res.iters[j])
        ts = int(v["cand_ts"][i])
        assert (keys[ts] if ts >= 0 else None) == (res.ts_list[res.ts[j]].key if res.ts[j] >= 0 else None)


@pytest.fixture(scope="module")
def qc2640():
    w = synth.workload("qc2640")
    v = run_lib(w["code"], **_params(w))
    return w, v


def test_qc2640_full_size_sampled(qc2640):
    w, v = qc2640
    g = _sampled_compare(w, v, 60, seed=5)
    assert v["info"]["girth"] == 8
    # the 8-cycle sets of size 4 are present
    assert (v["cand_vars"][:, 3] >= 0).sum() > 0
    _ts_invariants(g, v, qc=True)


def test_large_qc_code_variable_node_form_sampled():
    # n = 11520 (4 x 30 base, Z = 384, check degree up to 28): the two-buffer
    # layout of the two-codeword kernel does not fit a CTA, so the decode runs
    # its variable-node-pass form; sampled candidates against the oracle
    code = synth.batch_codes([122])[0]
    w = dict(code=code, K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)
    v = run_lib(code, cand_end=3000, **_params(w))
    assert len(v["cand_thr"]) == 3000
    rows = np.concatenate([(v["cand_vars"] >= 0).sum(1, keepdims=True), v["cand_vars"]], axis=1)
    rng = np.random.default_rng(3)
    pick = np.sort(rng.choice(len(rows), 30, replace=False))
    g = oracle.Graph(code)
    res = g.enumerate(rows[pick], **_params(w))
    assert (res.thr >= 0).any()
    for j, i in enumerate(pick):
        assert int(v["cand_thr"][i]) == int(res.thr[j]), rows[i]
        assert int(v["cand_decodes"][i]) == int(res.decodes[j]), rows[i]
        assert int(v["cand_iters"][i]) == int(res.iters[j]), rows[i]
        ts = int(v["cand_ts"][i])
        lkey = v["keys"][ts] if ts >= 0 else None
        okey = res.ts_list[res.ts[j]].key if res.ts[j] >= 0 else None
        assert lkey == okey, rows[i]
