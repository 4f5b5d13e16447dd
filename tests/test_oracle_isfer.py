"""Oracle pins for the importance-sampling FER estimator (mean-shift IS of
BPSK/AWGN toward a trapping set; Sec. II-III name Cole's weighting, the
formula is this library's reading).

Pinned by: mu = 0 giving weight 1 exactly (plain Monte Carlo), the
Gaussian moments of the Box-Muller normals, the series log / sin / cos
against double precision, the likelihood ratio recomputed in closed form,
and unbiasedness against plain Monte Carlo where both can be measured."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_series_log_and_sincos():
    for u in np.concatenate([np.geomspace(1e-7, 1 - 1e-7, 2000), [0.5, 0.25, 0.75]]).astype(np.float32):
        got, want = oracle.logf(u), math.log(float(u))
        assert abs(got - want) <= 3 * np.spacing(np.float32(abs(want))) + 1e-12, u
    for t in np.linspace(0, 1, 4001, endpoint=False).astype(np.float32):
        s, c = oracle.sincos2pi(t)
        assert abs(s - math.sin(2 * math.pi * float(t))) < 4e-7
        assert abs(c - math.cos(2 * math.pi * float(t))) < 4e-7


def test_box_muller_moments():
    g = np.concatenate([oracle.normals4(11, s, q) for s in range(500) for q in range(200)]).astype(np.float64)
    n = g.size  # 400,000 normals
    assert abs(g.mean()) < 5 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(((g - g.mean()) ** 4).mean() / g.var() ** 2 - 3.0) < 5 * math.sqrt(24.0 / n)
    assert abs((g > 1.96).mean() - 0.025) < 5 * math.sqrt(0.025 * 0.975 / n)


def test_philox_counters_distinct_and_uniform():
    outs = np.array([oracle.philox4x32_10([i, 0, 0, 0], [5, 9]) for i in range(4096)], dtype=np.uint64)
    assert len(np.unique(outs[:, 0])) == 4096
    bits = np.unpackbits(outs.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / math.sqrt(bits.size)


def _tiny():
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    res = g.enumerate(K=20, base_llr=16, amp_steps=10, max_size=2)
    t = min(res.ts_list, key=lambda t: (t.b / t.a, t.a))
    return g, list(t.key)


def test_mu_zero_is_plain_monte_carlo():
    g, T = _tiny()
    fail, logw = g.is_samples(T, ebn0_db=3.0, mu=0.0, job=1, n=300)
    assert (logw == 0.0).all()


def test_log_weight_closed_form():
    # log w = sum_{v in T} (mu n_v - mu^2/2) / sigma^2 with n_v = sigma g_v
    g, T = _tiny()
    ebn0, mu, job = 2.5, 0.8, 3
    fail, logw = g.is_samples(T, ebn0_db=ebn0, mu=mu, job=job, s0=17, n=5)
    s2 = 1.0 / (2 * 0.5 * 10 ** (ebn0 / 10))
    sig = np.float32(math.sqrt(s2))
    for i in range(5):
        want = 0.0
        for v in sorted(T):
            n = np.float32(sig * oracle.normals4(job, 17 + i, v // 4)[v % 4])
            want += (float(n) * mu - mu * mu / 2.0) / s2
        assert abs(logw[i] - want) <= 1e-12 * max(1.0, abs(want))


def test_unbiased_against_plain_monte_carlo():
    # at low Eb/N0 plain MC sees enough failures; the shifted estimator must agree
    g, T = _tiny()
    N = 6000
    f0, _ = g.is_samples(T, ebn0_db=1.0, mu=0.0, job=5, n=N)
    p0 = f0.mean()
    f1, lw1 = g.is_samples(T, ebn0_db=1.0, mu=0.6, job=6, n=N)
    w = f1 * np.exp(lw1)
    p1 = w.mean()
    se = math.sqrt(p0 * (1 - p0) / N + w.var() / N)
    assert p0 > 0.01
    assert abs(p1 - p0) < 5 * se, (p0, p1, se)


def test_quantizer_rounds_half_away_and_saturates():
    # 8 * LLR rounded half away from zero (round-to-even would give 2, -2, 0)
    for y, cq, sat, want in ((2.5, 1.0, 511, 3), (-2.5, 1.0, 511, -3), (0.5, 1.0, 511, 1), (-0.5, 1.0, 511, -1),
                             (1.5, 1.0, 511, 2), (0.4999999701976776, 1.0, 511, 0), (0.75, 2.0, 511, 2),
                             (600.0, 1.0, 511, 511), (-600.0, 1.0, 511, -511), (3.0, 2.0, 5, 5), (-3.0, 2.0, 5, -5)):
        assert oracle.is_quant(y, cq, sat) == want, (y, cq, sat)


@pytest.mark.parametrize("ebn0,mu,sat", [(4.0, 1.0, 511), (0.0, 0.7, 20)])
def test_channel_llr_from_the_definition(ebn0, mu, sat):
    # channel LLR 2 y / sigma^2 in units of 1/8 (x 16 / sigma^2), y = 1 + n - mu [v in T],
    # sigma^2 = 1 / (2 R Eb/N0), rounded half away from zero and saturated to +-sat;
    # recomputed here from the drawn normals, then decoded to the same fail flags
    g, T = _tiny()
    R = 1.0 - g.m / g.n
    s2 = 1.0 / (2.0 * R * 10.0 ** (ebn0 / 10.0))
    sig = np.float32(math.sqrt(s2))
    cq = np.float32(16.0 / s2)
    inT = np.zeros(g.n, bool)
    inT[list(T)] = True
    job = 21
    n_sat = 0
    for s in range(40):
        gn = np.concatenate([oracle.normals4(job, s, q) for q in range((g.n + 3) // 4)])[:g.n].astype(np.float32)
        n = (sig * gn).astype(np.float32)
        y = (np.float32(1.0) + n).astype(np.float32)
        y = np.where(inT, (y - np.float32(mu)).astype(np.float32), y)
        prod = (y * cq).astype(np.float32).astype(np.float64)
        want = np.clip(np.sign(prod) * np.floor(np.abs(prod) + 0.5), -sat, sat).astype(np.int32)
        L, nv = g.is_channel(T, ebn0_db=ebn0, mu=mu, job=job, sample=s, sat=sat)
        assert np.array_equal(nv, n)
        assert np.array_equal(L, want), s
        n_sat += int((np.abs(want) == sat).sum())
        fail, _ = g.is_samples(T, ebn0_db=ebn0, mu=mu, job=job, s0=s, n=1, sat=sat)
        f, *_ = g.decode_nms(want, K=20, sat=sat, wstart=1)
        assert bool(fail[0]) == f
    if sat < 100:
        assert n_sat > 0
