"""GPU parity of the importance-sampling FER estimator: per-sample failure
flags and log-weights bit-identical to the oracle (noise, quantization and
decoder are exact on both sides), estimates equal up to the order of the
double-precision sum; and the oracle's Philox generator against cuRAND's."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import paper_2208_05795_gb300 as tsx
import synth

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_equals_curand(tmp_path):
    so = str(tmp_path / "libcurandref.so")
    subprocess.check_call(["nvcc", "-shared", "-Xcompiler", "-fPIC", "-gencode", "arch=compute_103a,code=sm_103a",
                           "-o", so, os.path.join(HERE, "curand_philox_ref.cu")])
    lib = ctypes.CDLL(so)
    rng = np.random.default_rng(4)
    n = 2000
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:10] = 0
    ctr[10:20, 1:] = 0
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    key[:5] = 0
    out = np.zeros((n, 4), dtype=np.uint32)
    assert lib.curand_philox_ref(ctr.ctypes.data_as(ctypes.c_void_p), key.ctypes.data_as(ctypes.c_void_p),
                                 out.ctypes.data_as(ctypes.c_void_p), n) == 0
    for i in range(n):
        assert np.array_equal(oracle.philox4x32_10(ctr[i], key[i]), out[i]), i


def _first_ts(code, n_cand, **p):
    # the biased set T: the oracle's lowest-threshold trapping set over the
    # first n_cand canonical candidates (an input of both sides, so it comes
    # from the oracle)
    g = oracle.Graph(code)
    cands = g.candidates(p.get("max_size", 3), 0)[:n_cand]
    res = g.enumerate(cands, **p)
    t = min(res.ts_list, key=lambda t: (t.thr, t.a, t.key))
    return tsx.load_code(code), list(t.key)


@pytest.mark.parametrize("ebn0,mu", [(3.0, 1.0), (2.0, 0.0), (4.5, 0.7)])
def test_isfer_qc96_bit_exact(ebn0, mu):
    w = synth.workload("qc96")
    c, T = _first_ts(w["code"], 10**6, K=20, base_llr=16, amp_steps=10, max_size=2)
    N = 3000
    r = tsx.is_fer_estimate(c, T, ebn0_db=ebn0, mu=mu, n_samples=N, job_key=77, K=20, record=True)
    fail, logw = oracle.Graph(w["code"]).is_samples(T, ebn0_db=ebn0, mu=mu, job=77, n=N, K=20)
    assert np.array_equal(r["fail"], fail)
    assert np.array_equal(r["logw"], logw)
    if mu == 0.0:
        assert (r["logw"] == 0.0).all()
    want = float(np.sum(fail * np.exp(logw))) / N
    assert abs(r["fer"] - want) <= 1e-12 * max(want, 1e-300)
    assert r["n_fail"] == int(fail.sum()) and r["decodes"] == N


def test_isfer_peg1008_full_size_sampled():
    # 10^6 samples on the PEG code; a window of samples checked against the oracle
    w = synth.workload("peg1008")
    c, T = _first_ts(w["code"], 1100, K=w["K"], base_llr=16, amp_steps=w["amp_steps"], max_size=2)
    N = 1_000_000
    r = tsx.is_fer_estimate(c, T, ebn0_db=4.0, mu=1.0, n_samples=N, job_key=9, K=w["K"], record=True)
    assert r["n_samples"] == N and r["decodes"] == N
    g = oracle.Graph(w["code"])
    for s0 in (0, 654321):
        fail, logw = g.is_samples(T, ebn0_db=4.0, mu=1.0, job=9, s0=s0, n=200, K=w["K"])
        assert np.array_equal(r["fail"][s0:s0 + 200], fail)
        assert np.array_equal(r["logw"][s0:s0 + 200], logw)
    # a shard of the same job continues the same sample stream
    r2 = tsx.is_fer_estimate(c, T, ebn0_db=4.0, mu=1.0, n_samples=1000, sample_begin=654321, job_key=9,
                             K=w["K"], record=True)
    assert np.array_equal(r2["fail"], r["fail"][654321:655321])
    assert np.array_equal(r2["logw"], r["logw"][654321:655321])
    want = float(np.sum(r["fail"] * np.exp(r["logw"]))) / N
    assert abs(r["fer"] - want) <= 1e-9 * max(want, 1e-300)


def test_isfer_flat_form_full_size_sampled():
    # the n = 8,832 QC code (3 x 23 all-ones base, Z = 384, check degree 23):
    # the sampling kernel's all-row-block check pass with two checks a thread
    code = synth.serving_codes(2026, 8)[4]
    c, T = _first_ts(code, 40, K=20, base_llr=16, amp_steps=10, max_size=2)
    N = 200_000
    r = tsx.is_fer_estimate(c, T, ebn0_db=3.5, mu=1.0, n_samples=N, job_key=31, K=20, record=True)
    assert r["n_samples"] == N and 0 < r["fail"].sum() < N
    g = oracle.Graph(code)
    for s0 in (0, 123457, N - 60):
        fail, logw = g.is_samples(T, ebn0_db=3.5, mu=1.0, job=31, s0=s0, n=60, K=20)
        assert np.array_equal(r["fail"][s0:s0 + 60], fail), s0
        assert np.array_equal(r["logw"][s0:s0 + 60], logw), s0
