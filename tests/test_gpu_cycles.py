"""GPU parity of the cycle search (Sec. II, Prop. 1): the EMD spectrum of
Table II and the per-node 4- and 6-cycle counts of Table V, against the
paper's printed Code 1 values and the oracle."""
import multiprocessing as mp

import numpy as np
import pytest

import helpers
import oracle
import paper_2208_05795_gb300 as tsx
import synth

pytestmark = pytest.mark.gpu


def _code1():
    E, Z, extra = helpers.load_code1()
    return synth.qc_code(E, Z), extra


def _walks_job(args):
    code, v, lmax = args
    return oracle.Graph(code).cycle_walks(v, lmax, emd=True)


def _oracle_spectrum(code, lmax, starts):
    with mp.get_context("spawn").Pool(min(16, len(starts))) as pool:
        parts = pool.map(_walks_job, [(code, v, lmax) for v in starts])
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def test_code1_table2_up_to_12_cycles():
    code, _ = _code1()
    c = tsx.load_code(code)
    s = tsx.emd_spectrum(c, 6)
    # the oracle, walk for walk (its 12-cycle search is written by make_spectra.py)
    walks, hist = helpers.load_emd_golden()
    assert np.array_equal(s["count2l"][:7], hist)
    assert np.array_equal(s["walks"][2:7], walks[2:7])
    # Table II: rows 4 to 10 in full (printed rounded: 5380.5 as 5381); row 12
    # in full except EMD 2, 5 and 6, where closed chains made of two distinct
    # shorter cycles sharing a path are counted here and not in the table
    want = helpers.load_table2_code1()
    for (clen, e), count in want.items():
        l = clen // 2
        got = s["count2l"][l, e] / (2 * l)
        if clen == 12 and e in (2, 5, 6):
            assert got > count, (clen, e, got, count)
            continue
        assert got == count or got == count - 0.5, (clen, e, got, count)
    for l in range(2, 7):
        for e in np.flatnonzero(s["count2l"][l]):
            assert (2 * l, int(e)) in want, (2 * l, e)


@pytest.mark.parametrize("name,lmax", [("qc96", 6), ("peg1008", 5), ("qc2640", 6)])
def test_spectrum_equals_oracle(name, lmax):
    code = synth.workload(name)["code"]
    c = tsx.load_code(code)
    s = tsx.emd_spectrum(c, lmax)
    starts = [j * code.Z for j in range(code.n // code.Z)] if code.kind == "qc" else list(range(code.n))
    walks, hist = _oracle_spectrum(code, lmax, starts)
    assert np.array_equal(s["count2l"][:lmax + 1], hist)
    assert np.array_equal(s["walks"][:lmax + 1], walks)


@pytest.mark.parametrize("which", ["qc96", "peg1008", "code1", "batch"])
def test_node_cycle_counts(which):
    if which == "code1":
        code, extra = _code1()
    elif which == "batch":
        code = synth.batch_codes([122])[0]
    else:
        code = synth.workload(which)["code"]
    c = tsx.load_code(code)
    c4, c6 = tsx.cycle_counts(c)
    g = oracle.Graph(code)
    picks = range(code.n) if code.n <= 1100 else range(0, code.n, max(1, code.n // 300))
    for v in picks:
        w = g.cycle_walks(v, 3)
        assert (c4[v], c6[v]) == (w[2] // 2, w[3] // 2), v
    if which == "code1":
        from test_oracle_graph import _printed_matches
        for j in range(20):
            assert _printed_matches(c6[j * code.Z] / 3, extra["col_cyc6"][j])
            assert _printed_matches(c4[j * code.Z] / 2, extra["col_cyc4"][j])
