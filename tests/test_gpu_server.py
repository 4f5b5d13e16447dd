"""GPU: the serving runtime.

Every job's result must be the same alone and in the mix: an enumeration
job run by the server (chunked decode launches, a grid sized to its work,
other jobs on the device at the same time) gives exactly what enumerate_ts
gives for it alone, and an importance-sampling job exactly what
is_fer_estimate gives (same failures, same fixed-order sums).  Admission
must keep the admitted footprint within the budget.
"""
import numpy as np
import pytest

import synth
import paper_2208_05795_gb300 as tsx
from test_gpu_batch import _same

pytestmark = pytest.mark.gpu

ENUM = dict(K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)


@pytest.fixture(scope="module")
def mix():
    qc96 = synth.workload("qc96")["code"]
    codes = [qc96] + synth.batch_codes([102, 116]) + synth.serving_codes(7, 3)
    handles = [tsx.load_code(c) for c in codes]
    jobs = []
    for i, h in enumerate(handles):
        p = dict(ENUM, max_size=3) if i == 0 else dict(ENUM)
        if i >= 3:
            p["cand_end"] = 3000 + 1000 * i  # a job of a few thousand candidates
        jobs.append(("enum", h, tsx.make_params(**p)))
    # importance sampling toward the lowest-threshold set of the tiny code
    v0 = tsx.ts_list_view(tsx.enumerate_ts(handles[0], tsx.make_params(**dict(ENUM, max_size=3))))
    ts = v0["keys"][int(np.argmin(np.where(v0["thr"] >= 0, v0["thr"], 1 << 30)))]
    for k, (ebn0, mu) in enumerate([(3.0, 1.0), (4.0, 0.8), (5.0, 0.0)]):
        jobs.append(("is", handles[0], dict(ts_vars=ts, ebn0_db=ebn0, mu=mu, n_samples=50000, job_key=11 + k)))
    ts2 = tuple(range(0, 6 * 64, 64))[:3]  # three nodes of a larger code
    jobs.append(("is", handles[1], dict(ts_vars=ts2, ebn0_db=3.5, mu=1.0, n_samples=30000, job_key=5)))
    alone = []
    for kind, h, p in jobs:
        if kind == "enum":
            alone.append(tsx.ts_list_view(tsx.enumerate_ts(h, p)))
        else:
            q = dict(p)
            alone.append(tsx.is_fer_estimate(h, q.pop("ts_vars"), **q))
    return handles, jobs, alone


def _submit_all(srv, jobs):
    ids = []
    for kind, h, p in jobs:
        if kind == "enum":
            ids.append(srv.submit_enumerate(h, p))
        else:
            q = dict(p)
            ids.append(srv.submit_is_fer(h, q.pop("ts_vars"), **q))
    return ids


def _check_same(srv, jobs, ids, alone):
    for (kind, _, _), jid, ref in zip(jobs, ids, alone):
        r = srv.wait(jid)
        assert r["status"] == 0, r
        if kind == "enum":
            _same(srv.view(jid), ref)
        else:
            got = r["is_result"]
            for k in ("fer", "var", "sum_w", "sum_w2", "n_samples", "n_fail", "decodes", "iterations",
                      "edge_updates"):
                assert got[k] == ref[k], k


@pytest.mark.parametrize("serial", [0, 1])
def test_server_results_same_alone_and_in_mix(mix, serial):
    handles, jobs, alone = mix
    # small chunks so that every job is split into several launches
    with tsx.Server(max_jobs=4, serial=serial, chunk_candidates=2048, chunk_samples=8192) as srv:
        ids = _submit_all(srv, jobs)
        _check_same(srv, jobs, ids, alone)
        st = srv.stats()
        assert st["done"] == len(jobs) and st["failed"] == 0
        assert 0 < st["p50_ms"] <= st["p90_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["max_concurrent"] <= (1 if serial else 4)
        if not serial:
            assert st["max_concurrent"] >= 2
        for jid in ids:
            srv.release(jid)
        with pytest.raises(tsx.TsxError):
            srv.poll(ids[0])


def test_server_hbm_admission(mix):
    handles, jobs, alone = mix
    # a budget that holds the largest job but not all jobs at once
    with tsx.Server(max_jobs=8) as probe:
        ids = _submit_all(probe, jobs)
        sizes = [probe.wait(j)["device_bytes"] for j in ids]
    budget = max(sizes) + min(sizes)
    assert budget < sum(sizes)
    with tsx.Server(max_jobs=8, hbm_bytes=budget, chunk_candidates=4096) as srv:
        ids = _submit_all(srv, jobs)
        _check_same(srv, jobs, ids, alone)
        st = srv.stats()
        assert st["hbm_peak_bytes"] <= budget
        assert st["done"] == len(jobs)
    with tsx.Server(max_jobs=2, hbm_bytes=min(sizes)) as small:
        big = int(np.argmax(sizes))
        kind, h, p = jobs[big]
        with pytest.raises(tsx.TsxError):
            if kind == "enum":
                small.submit_enumerate(h, p)
            else:
                q = dict(p)
                small.submit_is_fer(h, q.pop("ts_vars"), **q)


def test_server_rejects_bad_jobs(mix):
    handles, _, _ = mix
    with tsx.Server() as srv:
        with pytest.raises(tsx.TsxError):
            srv.submit_enumerate(handles[0], tsx.make_params(**dict(ENUM, max_size=9)))
        with pytest.raises(tsx.TsxError):
            srv.submit_is_fer(handles[0], [10 ** 6], n_samples=10)
        jid = srv.submit_is_fer(handles[0], [0, 1, 2], n_samples=1000)
        assert srv.wait(jid)["status"] == 0


def test_server_timed_stream_with_list_and_budget_jobs(mix):
    # jobs arrive one by one (seeded exponential gaps) while others run, and the
    # mix includes an ordered-list job and a job with iteration budgets; each
    # result must still equal the stand-alone call's
    import time
    handles, jobs, alone = mix
    extra = [("enum", handles[0], tsx.make_params(**dict(ENUM, max_size=3, list_mode=1, kstart=-1))),
             ("enum", handles[1], tsx.make_params(**dict(ENUM, budget_wref=4, budget_kmin=5, cand_end=6000)))]
    extra_alone = [tsx.ts_list_view(tsx.enumerate_ts(h, p)) for _, h, p in extra]
    all_jobs, all_alone = jobs + extra, alone + extra_alone
    order = np.random.default_rng(17).permutation(len(all_jobs))
    gaps = np.random.default_rng(18).exponential(0.004, len(all_jobs))
    with tsx.Server(max_jobs=4, chunk_candidates=2048, chunk_samples=8192) as srv:
        ids = {}
        for k, g in zip(order, gaps):
            time.sleep(float(g))
            ids[k] = _submit_all(srv, [all_jobs[k]])[0]
        sel = sorted(ids)
        _check_same(srv, [all_jobs[k] for k in sel], [ids[k] for k in sel], [all_alone[k] for k in sel])
        st = srv.stats()
        assert st["done"] == len(all_jobs) and st["failed"] == 0
