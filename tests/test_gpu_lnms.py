"""GPU parity of the simulation decoder of Sec. III (quantized normalized
layered min-sum, 4/4/6 bits, 20 iterations), its frame-error simulation and
the generalized union bound, against the oracle: per frame the same failure
flag, iteration count and decision; the union bound equal to the oracle's
sum of importance-sampling estimates."""
import math
import zlib

import numpy as np
import pytest

import helpers
import oracle
import paper_2208_05795_gb300 as tsx
import synth

pytestmark = pytest.mark.gpu


def _codes():
    E, Z, _ = helpers.load_code1()
    return {"qc96": synth.workload("qc96")["code"], "code1": synth.qc_code(E, Z),
            "batch103": synth.batch_codes([103])[0]}


@pytest.mark.parametrize("name", ["qc96", "code1", "batch103"])
@pytest.mark.parametrize("widths", [(4, 4, 6, 20), (5, 5, 7, 8), (3, 4, 5, 20)])
def test_lnms_decode_bit_exact(name, widths):
    import torch
    code = _codes()[name]
    lb, cb, vb, K = widths
    g = oracle.Graph(code)
    rng = np.random.default_rng(zlib.crc32(repr((name, widths)).encode()))
    nf = 300
    lim = (1 << (lb - 1)) - 1
    # frames around +3 at three noise levels (most decode at the lowest, few at the highest), with values
    # beyond the LLR width on both sides (saturated)
    sd = np.array([1.0, 2.0, 3.0])[np.arange(nf) % 3][:, None]
    llr = np.clip(np.round(rng.normal(3.0, 1.0, (nf, g.n)) * sd + 3.0 * (1 - sd)), -100, 100).astype(np.int8)
    d = torch.from_numpy(llr).cuda()
    fail = torch.zeros(nf, dtype=torch.uint8, device="cuda")
    it = torch.zeros(nf, dtype=torch.int32, device="cuda")
    x = torch.zeros((nf, g.n), dtype=torch.uint8, device="cuda")
    c = tsx.load_code(code)
    tsx.lnms_decode(c, d.data_ptr(), nf, fail.data_ptr(), it.data_ptr(), x.data_ptr(), K=K, llr_bits=lb,
                    c2v_bits=cb, v2c_bits=vb)
    torch.cuda.synchronize()
    fail, it, x = fail.cpu().numpy(), it.cpu().numpy(), x.cpu().numpy()
    nfail, bad = 0, []
    for f in range(nf):
        of, ox, ok = g.decode_lnms(llr[f].astype(np.int32), K=K, llr_bits=lb, c2v_bits=cb, v2c_bits=vb)
        if (bool(fail[f]), int(it[f])) != (of, ok) or not np.array_equal(x[f], ox):
            bad.append((f, bool(fail[f]), int(it[f]), of, ok, int((x[f] != ox).sum())))
        nfail += of
    assert not bad, (len(bad), bad[:8])
    assert 0 < nfail < nf
    assert lim >= 3


def test_simulation_frames_bit_exact_and_stop_rule():
    code = _codes()["code1"]
    g = oracle.Graph(code)
    c = tsx.load_code(code)
    kw = dict(ebn0_db=2.75, llr_scale=1.0, job_key=77, frame_begin=5)
    r = tsx.lnms_simulate(c, max_frames=2000, max_errors=0, record=True, **kw)
    of, oit, ow = g.lnms_frames(ebn0_db=2.75, llr_scale=1.0, job=77, f0=5, n=2000)
    assert r["frames"] == 2000
    assert np.array_equal(r["fail"], of)
    assert r["frame_errors"] == int(of.sum()) > 5
    assert r["bit_errors"] == int(ow[of > 0].sum())
    assert r["iterations"] == int(oit.sum())
    assert r["edge_updates"] == int(oit.sum()) * g.E
    # stop at the frame that brings the errors to 5
    r5 = tsx.lnms_simulate(c, max_frames=2000, max_errors=5, **kw)
    assert r5["frames"] == int(np.flatnonzero(of)[4]) + 1 and r5["frame_errors"] == 5


def test_union_bound_equals_oracle_sum():
    w = synth.workload("qc96")
    code = w["code"]
    g = oracle.Graph(code)
    res = g.enumerate(K=20, base_llr=16, amp_steps=10, max_size=2)
    sets = sorted(res.ts_list, key=lambda t: (t.thr, t.a, t.key))[:5]
    c = tsx.load_code(code)
    kw = dict(ebn0_db=2.0, mu=1.0, n_samples=3000, job_key=500, K=20)
    u = tsx.union_bound_fer(c, [t.key for t in sets], [t.orbit for t in sets], **kw)
    want, var = 0.0, 0.0
    for i, t in enumerate(sets):
        fail, logw = g.is_samples(t.key, ebn0_db=2.0, mu=1.0, job=500 + i, n=3000, K=20)
        wv = fail * np.exp(logw)
        fer = wv.mean()
        assert math.isclose(u["fer"][i], fer, rel_tol=1e-9, abs_tol=1e-300), i
        want += t.orbit * fer
        var += t.orbit ** 2 * ((wv ** 2).mean() - fer ** 2) / 3000
    assert math.isclose(u["fer_ub"], want, rel_tol=1e-9)
    assert math.isclose(u["var_ub"], var, rel_tol=1e-6)
    assert u["n_sets"] == 5 and u["samples"] == 15000 and want > 0
