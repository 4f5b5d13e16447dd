"""Shared test helpers: golden-file loaders and small independent graph tools.

Nothing here implements the method under test; the graph tools below
(adjacency lists, cycle enumeration, distances) are written separately from
both the oracle and the CUDA library so that they can cross-check them.
"""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def load_code1():
    """Table V: Code 1 exponent matrix and its Cyc4/Cyc6 averages."""
    Z, rows, extra = None, [], {}
    for tok in _rows("code1_table5.txt"):
        if tok[0] == "Z":
            Z = int(tok[1])
        elif tok[0] in ("col_cyc6", "col_cyc4", "row_cyc6", "row_cyc4"):
            extra[tok[0]] = tok[1:]
        else:
            rows.append([int(x) for x in tok])
    return np.array(rows, dtype=np.int32), Z, extra


def load_table2_code1():
    return {(int(a), int(b)): int(c) for a, b, c in _rows("code1_table2_emd.txt")}


def load_table3_code1():
    return {(int(a), int(b)): int(c) for a, b, c in _rows("code1_table3_ts.txt")}


def dense_qc(shifts, Z):
    """H from the exponent matrix written straight from eq. 1: block P^a has
    P_{r,c} = 1 iff c = r + a (mod Z)."""
    m_b, n_b = shifts.shape
    H = np.zeros((m_b * Z, n_b * Z), dtype=np.uint8)
    eye = np.eye(Z, dtype=np.uint8)
    for i in range(m_b):
        for j in range(n_b):
            a = int(shifts[i, j])
            if a >= 0:
                H[i * Z:(i + 1) * Z, j * Z:(j + 1) * Z] = np.roll(eye, a, axis=1)
    return H


def adjacency(H):
    vn = [list(np.flatnonzero(H[:, v])) for v in range(H.shape[1])]
    cn = [list(np.flatnonzero(H[c])) for c in range(H.shape[0])]
    return vn, cn


def cycles_through_vn(vn, cn, v0, l):
    """All simple cycles of length 2l through variable node v0, each once,
    as (list of VNs, list of checks) in walk order."""
    out = {}
    v0_checks = set(vn[v0])

    def rec(vs, cs):
        v = vs[-1]
        if len(vs) == l:
            for c in vn[v]:
                if c in v0_checks and c not in cs and (l > 1 or True):
                    cc = cs + [c]
                    if len(set(cc)) == len(cc):
                        out[_cyc_key(vs, cc)] = (list(vs), cc)
            return
        for c in vn[v]:
            if c in cs:
                continue
            for u in cn[c]:
                if u == v or u in vs:
                    continue
                rec(vs + [u], cs + [c])

    rec([v0], [])
    return list(out.values())


def _cyc_key(vs, cs):
    # a cycle is determined by its alternating node sequence up to rotation/reflection
    seq = []
    for v, c in zip(vs, cs):
        seq += [("v", int(v)), ("c", int(c))]
    n = len(seq)
    rots = []
    for s in range(0, n, 2):
        r = seq[s:] + seq[:s]
        rots.append(tuple(r))
        rr = [r[0]] + r[1:][::-1]
        rots.append(tuple(rr))
    return min(rots)


def emd(cn_sets, H, vs):
    """Extrinsic message degree: checks adjacent to exactly one VN of the set."""
    cnt = H[:, sorted(vs)].sum(axis=1)
    return int((cnt == 1).sum())


def load_emd_golden(name="emd_code1_l6.txt"):
    """The oracle's EMD spectrum file (make_spectra.py code1_emd): walks[l] and count2l[l, e]."""
    walks = np.zeros(7, dtype=np.int64)
    hist = np.zeros((7, 128), dtype=np.int64)
    for tok in _rows(name):
        if tok[0] == "walks":
            walks[int(tok[1])] = int(tok[2])
        else:
            hist[int(tok[0]), int(tok[1])] = int(tok[2])
    return walks, hist
