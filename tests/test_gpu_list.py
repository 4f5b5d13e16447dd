"""GPU parity of the ordered list of Sec. III (every non-empty S1(x_k),
S2(x_k), k = kstart .. K_last, of the decode at the threshold, run as the
second stage over the failing candidates) and of the cycle-density iteration
budgets, against the oracle: bit-exact trapping-set lists (key, a, b, orbit,
count, minimum threshold, elementary flag, which sieves reached the set) and
per-candidate thresholds, decodes and iterations."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib_cand_tuples, run_lib

pytestmark = pytest.mark.gpu


def _params(w, **over):
    p = dict(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"], max_size=w["max_size"],
             cycle_len=w["cycle_len"])
    p.update(over)
    return p


def _rows(v):
    cv = v["cand_vars"]
    return np.concatenate([(cv >= 0).sum(1, keepdims=True), cv], axis=1).astype(np.int32)


def _compare_list(v, res):
    got = {k: (int(a), int(b), int(o), int(c), int(t), int(f) & 1, (int(f) >> 1) & 3)
           for k, a, b, o, c, t, f in zip(v["keys"], v["a"], v["b"], v["orbit"], v["count"], v["thr"], v["flags"])}
    want = {t.key: (t.a, t.b, t.orbit, t.count, t.thr, int(t.elementary), t.kind) for t in res.ts_list}
    assert got.keys() == want.keys(), (len(got), len(want))
    bad = [k for k in want if got[k] != want[k]]
    assert not bad, [(k, got[k], want[k]) for k in bad[:5]]
    assert np.array_equal(v["cand_thr"], res.thr)
    assert np.array_equal(v["cand_decodes"], res.decodes)
    assert np.array_equal(v["cand_iters"], res.iters)
    assert (v["cand_ts"] == -1).all()


@pytest.mark.parametrize("kstart", [0, -1, 7])
def test_qc96_list_mode_bit_exact(kstart):
    w = synth.workload("qc96")
    p = _params(w, list_mode=1, kstart=kstart)
    v = run_lib(w["code"], **p)
    g = oracle.Graph(w["code"])
    res = g.enumerate(_rows(v), **{k: x for k, x in p.items() if k not in ("list_mode",)}, list_mode=True)
    _compare_list(v, res)
    s = v["stats"]
    want_ks = {0: 3, 7: 7}.get(kstart, res.kstart)
    assert s["list_kstart"] == want_ks
    assert (s["converged"], s["converged_iterations"]) == (res.converged, res.converged_iterations)
    assert len(v["keys"]) > 300 and s["list_patterns"] > 0


@pytest.mark.parametrize("name,n", [("peg1008", 1200), ("qc2640", 150)])
def test_list_mode_shard_bit_exact(name, n):
    # a range of the full-size workloads' candidates, two-stage window start
    w = synth.workload(name)
    p = _params(w, list_mode=1, kstart=-1, cand_begin=0, cand_end=n)
    v = run_lib(w["code"], **p)
    assert len(v["cand_thr"]) == n
    g = oracle.Graph(w["code"])
    q = {k: x for k, x in p.items() if k not in ("list_mode", "cand_begin", "cand_end")}
    res = g.enumerate(_rows(v), **q, list_mode=True)
    _compare_list(v, res)
    assert v["stats"]["list_kstart"] == res.kstart


@pytest.mark.parametrize("kernel", [1, 2])
def test_iteration_budgets_bit_exact(kernel):
    # qc96 and a code with 4-cycles: candidates get kmin .. K iterations by their
    # nodes' cycle density; the two-codeword kernel carries a limit per half
    for code in (synth.workload("qc96")["code"],
                 synth.qc_code([[0, 1, 2, 3, 4, 5], [0, 2, 4, 6, 8, 10], [0, 3, 6, 1, 12, 15]], 16)):
        p = dict(K=20, base_llr=16, amp_steps=10, max_size=3, cycle_len=0, budget_wref=6, budget_kmin=4)
        v = run_lib(code, kernel=kernel, **p)
        g = oracle.Graph(code)
        res = g.enumerate(_rows(v), **p)
        assert np.array_equal(v["cand_thr"], res.thr)
        assert np.array_equal(v["cand_decodes"], res.decodes)
        assert np.array_equal(v["cand_iters"], res.iters)
        got = sorted((k, int(a), int(b), int(c), int(t)) for k, a, b, c, t in
                     zip(v["keys"], v["a"], v["b"], v["count"], v["thr"]))
        want = sorted((t.key, t.a, t.b, t.count, t.thr) for t in res.ts_list)
        assert got == want


def test_iteration_budget_peg_shard():
    w = synth.workload("peg1008")
    p = _params(w, budget_wref=4, budget_kmin=10, cand_begin=1000, cand_end=4000)
    v = run_lib(w["code"], **p)
    g = oracle.Graph(w["code"])
    q = {k: x for k, x in p.items() if k not in ("cand_begin", "cand_end")}
    res = g.enumerate(_rows(v), **q)
    assert np.array_equal(v["cand_thr"], res.thr)
    assert np.array_equal(v["cand_iters"], res.iters)
