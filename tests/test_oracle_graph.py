"""Oracle pins: Tanner-graph expansion (eqs. 1-2), girth and the Tanner ball.

Pinned to the paper's own numbers for Code 1 (Tables II and V) and to
hand-checked small graphs.
"""
from collections import Counter

import numpy as np
import pytest

import helpers
import oracle
import synth


def test_eq1_circulant_shifts_right():
    # eq. 1: P_ij = 1 iff i + 1 = j (mod L); P^k shifts I right k times.
    L = 5
    g = oracle.Graph(synth.qc_code([[1]], L))
    H = g.dense()
    for i in range(L):
        for j in range(L):
            assert H[i, j] == (1 if (i + 1) % L == j else 0)
    g3 = oracle.Graph(synth.qc_code([[3]], L))
    assert np.array_equal(g3.dense(), np.linalg.matrix_power(H.astype(int), 3).astype(np.uint8))


def test_zero_block():
    g = oracle.Graph(synth.qc_code([[0, -1], [2, 1]], 4))
    H = g.dense()
    assert H[:4, 4:].sum() == 0
    assert g.E == 3 * 4


def test_code1_size_and_circulants():
    E, Z, _ = helpers.load_code1()
    g = oracle.Graph(synth.qc_code(E, Z))
    # "77 non-zero circulants" (Sec. III, memory remark) -> 77 * 128 edges
    assert (E >= 0).sum() == 77
    assert g.n == 20 * 128 and g.m == 4 * 128 and g.E == 77 * 128
    assert np.array_equal(g.dense(), helpers.dense_qc(E, Z))


def test_code1_girth_is_4():
    # Table III caption: Code 1 has Girth = 4
    E, Z, _ = helpers.load_code1()
    assert oracle.Graph(synth.qc_code(E, Z)).girth() == 4


@pytest.fixture(scope="module")
def code1_adj():
    E, Z, extra = helpers.load_code1()
    g = oracle.Graph(synth.qc_code(E, Z))
    H = g.dense()
    vn, cn = helpers.adjacency(H)
    return H, vn, cn, Z, extra


def test_code1_emd_spectrum_table2(code1_adj):
    # Table II, Code 1 column, cycles of length 4 and 6, counted per orbit
    H, vn, cn, Z, _ = code1_adj
    want = helpers.load_table2_code1()
    got = Counter()
    for l in (2, 3):
        for j in range(20):
            for vs, _cs in helpers.cycles_through_vn(vn, cn, j * Z, l):
                got[(2 * l, helpers.emd(None, H, vs))] += 1
    for (clen, e), count in want.items():
        if clen <= 6:
            assert got[(clen, e)] / (clen // 2) == count, (clen, e)


def _printed_matches(x, printed):
    digits = len(printed.split(".")[1]) if "." in printed else 0
    val = float(printed)
    trunc = np.floor(x * 10 ** digits + 1e-9) / 10 ** digits
    return abs(round(x, digits) - val) < 1e-9 or abs(trunc - val) < 1e-9


def test_code1_cycle_density_table5(code1_adj):
    # Table V: average number of 4-/6-cycles through a column block, i.e.
    # cycles through VN (j,0) divided by the cycle's number of VNs (...)/2, /3
    H, vn, cn, Z, extra = code1_adj
    for j in range(20):
        c6 = len(helpers.cycles_through_vn(vn, cn, j * Z, 3))
        c4 = len(helpers.cycles_through_vn(vn, cn, j * Z, 2))
        assert _printed_matches(c6 / 3, extra["col_cyc6"][j]), (j, c6)
        assert _printed_matches(c4 / 2, extra["col_cyc4"][j]), (j, c4)
    # rows: cycles through check (i,0); walk from its VNs and keep those using it
    for i in range(4):
        c = i * Z
        cyc = {3: set(), 2: set()}
        for v0 in cn[c]:
            for l in (2, 3):
                for vs, cs in helpers.cycles_through_vn(vn, cn, v0, l):
                    if c in cs:
                        cyc[l].add(helpers._cyc_key(vs, cs))
        assert _printed_matches(len(cyc[3]) / 3, extra["row_cyc6"][i]), (i, len(cyc[3]))
        assert _printed_matches(len(cyc[2]) / 2, extra["row_cyc4"][i]), (i, len(cyc[2]))


def test_girth_small_cases():
    # a 2x2 all-zero-shift base has 4-cycles; a single 6-cycle graph has girth 6;
    # a tree has none
    assert oracle.Graph(synth.qc_code([[0, 0], [0, 0]], 3)).girth() == 4
    six = synth.csr_code(3, 3, [0, 2, 4, 6], [0, 1, 1, 2, 0, 2])
    assert oracle.Graph(six).girth() == 6
    tree = synth.csr_code(5, 2, [0, 3, 6], [0, 1, 2, 2, 3, 4])
    assert oracle.Graph(tree).girth() == 0


@pytest.mark.parametrize("name,g", [("qc96", 6), ("qc2640", 8)])
def test_workload_girth(name, g):
    w = synth.workload(name)
    assert oracle.Graph(w["code"]).girth() == g


def test_ball4_against_distances():
    # Tanner ball = VNs at graph distance 2 or 4, from an all-pairs BFS on H
    w = synth.workload("qc96")
    g = oracle.Graph(w["code"])
    H = g.dense().astype(np.int64)
    A = (H.T @ H > 0).astype(np.int64)  # VN-VN adjacency through a check
    np.fill_diagonal(A, 0)
    reach2 = A > 0
    reach4 = (A @ A > 0) | reach2
    for v in (0, 17, 95):
        want = set(np.flatnonzero(reach4[v])) - {v}
        assert set(g.ball4(v).tolist()) == want
