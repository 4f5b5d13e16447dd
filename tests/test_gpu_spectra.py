"""GPU parity at full size: whole trapping-set spectra against the oracle.

The expected values come from ``tests/golden/make_spectra.py``, which runs
only the oracle: every canonical candidate of the 2640-node QC code, and
the candidates of the first representatives of the 1008-node PEG code (at
least 200,000, the first ones of the library's candidate order, decoded by
the library as the range [0, N)).  Everything is compared element by
element: the candidate sets, per candidate the threshold amplitude, the
number of decodes and iterations, the sieve used and the trapping set
reached, and per distinct trapping set (a, b), canonical key, orbit size,
count, minimum threshold, elementary flag and the union of the sieves that
reached it.

The float decoder is also compared with the oracle's other reading of it
(the C library's tanhf / atanhf instead of the shared series): thresholds
within 1e-3, and the same trapping set wherever the thresholds agree.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib_cand_tuples, lib_records, oracle_cand_tuples, oracle_records, run_lib

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with np.load(os.path.join(GOLDEN, f"spectrum_{name}.npz")) as f:
        z = {k: f[k] for k in f.files}  # each access of the archive decompresses again: read once
    meta = json.loads(str(z["meta"]))
    flat, off = z["keys"].tolist(), z["key_off"].tolist()
    keys = [tuple(flat[off[i]:off[i + 1]]) for i in range(len(z["ts_a"]))]
    return z, meta, keys


def _params(meta, **over):
    p = {k: meta[k] for k in ("K", "base_llr", "amp_steps", "max_size", "cycle_len")}
    p.update(over)
    return p


def _compare(v, z, keys):
    cand = oracle_cand_tuples(z["cands"])
    assert sorted(lib_cand_tuples(v)) == sorted(cand)
    want = {}
    for i, t in enumerate(cand):
        ts = int(z["ts"][i])
        want[t] = (int(z["thr"][i]), keys[ts] if ts >= 0 else None, int(z["which"][i]), int(z["decodes"][i]),
                   int(z["iters"][i]))
    got = {t: (r[0], r[2], r[3], r[4], r[5]) for t, r in lib_records(v).items()}
    bad = [t for t in want if got[t] != want[t]]
    assert not bad, (len(bad), bad[:5], [(got[t], want[t]) for t in bad[:5]])
    # the distinct trapping sets
    assert v["keys"] == keys
    for f in ("a", "b", "orbit", "count", "thr"):
        assert np.array_equal(v[f], z["ts_" + f]), f
    assert np.array_equal(v["flags"] & 1, z["ts_elem"])
    union = np.zeros(len(keys), np.int32)
    np.bitwise_or.at(union, z["ts"][z["ts"] >= 0], (z["which"][z["ts"] >= 0] & 3) << 1)
    assert np.array_equal(v["flags"] & 6, union)


def test_qc2640_whole_spectrum_bit_exact():
    z, meta, keys = _golden("qc2640")
    w = synth.workload("qc2640")
    v = run_lib(w["code"], **_params(meta))
    assert v["stats"]["n_cand"] == meta["n_cand"] == len(z["cands"])
    _compare(v, z, keys)


def test_peg1008_shard_spectrum_bit_exact():
    z, meta, keys = _golden("peg1008_shard")
    w = synth.workload("peg1008")
    n = meta["n_cand"]
    v = run_lib(w["code"], cand_begin=0, cand_end=n, **_params(meta))
    assert v["stats"]["n_cand"] == n and v["stats"]["n_cand_total"] == meta["n_cand_code"]
    _compare(v, z, keys)


def test_spa_against_the_libm_reading():
    # the decoder's tanh/atanh read as any correct implementation: thresholds
    # within the stated 1e-3, the trapping set the same where they agree
    w = synth.workload("qc96")
    p = dict(K=w["K"], base_llr=w["base_llr"], amp_steps=12, max_size=w["max_size"], cycle_len=w["cycle_len"])
    v = run_lib(w["code"], decoder="spa", **p)
    g = oracle.Graph(w["code"])
    res = g.enumerate(decoder="spa", spa_libm=True, **p)
    lr, orr = lib_records(v), oracle_records(res)
    assert lr.keys() == orr.keys()
    same_thr = 0
    for t, rec in orr.items():
        assert abs(lr[t][1] - rec[1]) <= 1e-3, (t, lr[t], rec)
        if lr[t][1] == rec[1]:
            same_thr += 1
            assert lr[t][2] == rec[2], t
    assert same_thr > 0.5 * len(orr)
    # the sets reached by candidates whose thresholds agree are on both lists
    agree = {lr[t][2] for t, rec in orr.items() if lr[t][1] == rec[1] and rec[2] is not None}
    assert agree <= set(v["keys"]) and agree <= {t.key for t in res.ts_list}
