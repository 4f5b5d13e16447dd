"""Oracle pins for the paper's simulation decoder (Sec. III, Fig. 2):
quantized normalized layered min-sum with 4-bit channel LLRs, 4-bit
check-to-variable and 6-bit variable-to-check messages.

Pinned by a two-layer iteration worked by hand, by the saturation of each
width changing a decision the way the arithmetic says, by a QC row-block
layer giving the same result as its rows taken one at a time (its checks
touch distinct variable nodes), and by codeword inputs stopping at once."""
import numpy as np

import oracle
import synth


def _csr(n, rows):
    rp = np.cumsum([0] + [len(r) for r in rows])
    ci = np.concatenate([np.sort(np.array(r, dtype=np.int32)) for r in rows])
    return synth.csr_code(n, len(rows), rp, ci)


def test_two_layers_by_hand():
    # c0 = {0,1,2}, c1 = {2,3}; L = (5, -3, 2, 7), alpha 3/4.
    # iteration 1, layer c0: q = (5, -3, 2); r = (-1, +1, -2); P = (4, -2, 0, 7)
    #              layer c1: q = (0, 7);  r = (+5, 0);      P = (4, -2, 5, 7)
    #   x = (0, 1, 0, 0): c0 unsatisfied.
    # iteration 2, layer c0: q = (5, -3, 7); r = (-2, +3, -2); P = (3, 0, 5, 7)
    #              layer c1: q = (0, 7);  r = (+5, 0);      P = (3, 0, 5, 7)
    #   x = 0: stop after 2 iterations.
    g = oracle.Graph(_csr(4, [[0, 1, 2], [2, 3]]))
    L = [5, -3, 2, 7]
    f, x, kl = g.decode_lnms(L, K=1)
    assert f and x.tolist() == [0, 1, 0, 0] and kl == 1
    f, x, kl = g.decode_lnms(L, K=20)
    assert not f and x.tolist() == [0, 0, 0, 0] and kl == 2


def test_widths_saturate():
    g = oracle.Graph(_csr(2, [[0, 1]]))
    # LLR width 8 keeps L = (100, -10); q0 = sat6(100) = 31; r1 = (3 * 31) >> 2 = 23,
    # saturated to 7 at 4 bits: P1 = -10 + 7 = -3 < 0 (still failing)
    f, x, _ = g.decode_lnms([100, -10], K=1, llr_bits=8)
    assert f and x.tolist() == [0, 1]
    # with 6-bit check-to-variable messages r1 = 23 and P1 = 13: decoded
    f, x, _ = g.decode_lnms([100, -10], K=1, llr_bits=8, c2v_bits=6)
    assert not f and x.tolist() == [0, 0]
    # 4-bit channel LLRs: 100 and 7 are the same input
    assert g.decode_lnms([100, -3], K=3)[1].tolist() == g.decode_lnms([7, -3], K=3)[1].tolist()


def test_qc_row_block_layer_equals_its_rows():
    w = synth.workload("qc96")
    qc = oracle.Graph(w["code"])
    H = qc.dense()
    rows = [list(np.flatnonzero(H[c])) for c in range(H.shape[0])]
    gen = oracle.Graph(_csr(H.shape[1], rows))
    rng = np.random.default_rng(5)
    for t in range(20):
        # mostly reliable bits, some unreliable or wrong
        L = np.where(rng.random(qc.n) < 0.85, rng.integers(2, 8, qc.n), rng.integers(-7, 8, qc.n)).astype(np.int32)
        a = qc.decode_lnms(L, K=20)
        b = gen.decode_lnms(L, K=20)
        assert a[0] == b[0] and a[2] == b[2] and np.array_equal(a[1], b[1]), t


def test_codeword_inputs_stop_at_once():
    # every check satisfied by the hard decisions of L: no iteration runs
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    f, x, kl = g.decode_lnms(np.full(g.n, 3, np.int32), K=20)
    assert not f and kl == 0 and not x.any()
    # the planted weight-4 codeword of a small code, as the sign pattern of L
    code = _csr(6, [[0, 1, 4], [1, 2, 5], [2, 3, 4], [3, 0, 5], [0, 2]])
    g = oracle.Graph(code)
    L = np.array([-5, -5, -5, -5, 6, 6], np.int32)  # x = (1,1,1,1,0,0) satisfies every check
    f, x, kl = g.decode_lnms(L, K=20)
    assert f and kl == 0 and x.tolist() == [1, 1, 1, 1, 0, 0]


def test_simulation_channel_from_the_definition():
    # frame f: y = 1 + sigma g (g the importance-sampling generator's normals of
    # sample f), channel value round-half-away(2 y / sigma^2 * scale) saturated to
    # the LLR width; decoding those values gives the simulation's flags
    import math
    code = synth.workload("qc96")["code"]
    g = oracle.Graph(code)
    ebn0, scale, job = 2.0, 0.75, 9
    R = 1.0 - g.m / g.n
    s2 = 1.0 / (2.0 * R * 10 ** (ebn0 / 10))
    sig, cq = np.float32(math.sqrt(s2)), np.float32(2.0 * scale / s2)
    fail, it, w = g.lnms_frames(ebn0_db=ebn0, llr_scale=scale, job=job, f0=100, n=60)
    n_sat = 0
    for i in range(60):
        gn = np.concatenate([oracle.normals4(job, 100 + i, q) for q in range((g.n + 3) // 4)])[:g.n].astype(np.float32)
        y = (np.float32(1.0) + (sig * gn).astype(np.float32)).astype(np.float32)
        prod = (y * cq).astype(np.float32).astype(np.float64)
        L = np.clip(np.sign(prod) * np.floor(np.abs(prod) + 0.5), -7, 7).astype(np.int32)
        n_sat += int((np.abs(L) == 7).sum())
        f, x, kl = g.decode_lnms(L, K=20)
        assert (bool(fail[i]), int(it[i]), int(w[i])) == (f, kl, int(x.sum())), i
    assert n_sat > 0 and fail.any()
