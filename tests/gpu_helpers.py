"""Helpers of the GPU parity tests: run the CUDA library through its C ABI
and put its results and the oracle's side by side."""
import numpy as np

import paper_2208_05795_gb300 as tsx


def run_lib(code, **params):
    c = tsx.load_code(code)
    lst = tsx.enumerate_ts(c, **params)
    v = tsx.ts_list_view(lst)
    v["info"] = c.info
    return v


def lib_cand_tuples(v):
    out = []
    for r in v["cand_vars"]:
        out.append(tuple(int(x) for x in r if x >= 0))
    return out


def oracle_cand_tuples(cands):
    return [tuple(int(x) for x in r[1:1 + r[0]]) for r in cands]


def lib_records(v):
    """candidate tuple -> (thr, thr_f, ts key or None, sieve, decodes, iters)"""
    keys = v["keys"]
    rec = {}
    for i, t in enumerate(lib_cand_tuples(v)):
        ts = int(v["cand_ts"][i])
        rec[t] = (int(v["cand_thr"][i]), float(v["cand_thr_f"][i]), keys[ts] if ts >= 0 else None,
                  int(v["cand_flags"][i]) & 3, int(v["cand_decodes"][i]), int(v["cand_iters"][i]))
    return rec


def oracle_records(res):
    rec = {}
    for i, t in enumerate(oracle_cand_tuples(res.cands)):
        ts = int(res.ts[i])
        rec[t] = (int(res.thr[i]), float(res.thr_f[i]), res.ts_list[ts].key if ts >= 0 else None,
                  int(res.which[i]), int(res.decodes[i]), int(res.iters[i]))
    return rec


def lib_ts(v):
    """key -> (a, b, orbit, count, thr, thr_f, elementary)"""
    out = {}
    for i, k in enumerate(v["keys"]):
        out[k] = (int(v["a"][i]), int(v["b"][i]), int(v["orbit"][i]), int(v["count"][i]),
                  int(v["thr"][i]), float(v["thr_f"][i]), bool(v["flags"][i] & 1))
    return out


def oracle_ts(res):
    return {t.key: (t.a, t.b, t.orbit, t.count, t.thr, float(t.thr_f), t.elementary) for t in res.ts_list}
