"""Seeded QC-LDPC and PEG parity-check matrices shaped like the paper's workloads.

Conventions (paper Sec. II, eqs. 1-3): a QC code is given by its exponent
matrix E(H) of size m_b x n_b over {-1, 0, ..., Z-1}; -1 is the zero block
P^inf.  Nothing here decodes or classifies anything.

Recipes (all deterministic in the seed):

* ``draw_qc``: ``numpy.random.default_rng(seed).integers(0, Z, (m_b, n_b))``
  drawn whole, with -1 written where the base mask is 0, redrawn whole until
  the Tanner graph's girth is at least ``girth_min`` (checked by a
  breadth-first search that is local to this module).
* ``peg``: progressive edge growth (Hu, Eleftheriou, Arnold) for a
  (dv, dc)-regular graph: variable nodes are connected in index order; the
  first edge of a node goes to a check of minimum current degree, later
  edges to a check outside the breadth-first neighbourhood of the node, or
  first reached at its deepest level; among those the minimum current
  degree wins; checks already at degree dc are never chosen; remaining ties
  are broken by the seeded generator.
* ``batch_codes``: the 32 codes of the batching workload (seeds 100..131).
* ``serving_codes``: codes for the serving stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Code:
    """A parity-check matrix, either QC (exponent matrix) or general (CSR rows)."""

    kind: str  # "qc" or "csr"
    n: int
    m: int
    Z: int = 0
    shifts: Optional[np.ndarray] = None  # int32 [m_b, n_b], -1 = zero block
    row_ptr: Optional[np.ndarray] = None  # int32 [m+1] (csr)
    col_idx: Optional[np.ndarray] = None  # int32 [E]   (csr), ascending per row
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m_b(self) -> int:
        return int(self.shifts.shape[0]) if self.kind == "qc" else 0

    @property
    def n_b(self) -> int:
        return int(self.shifts.shape[1]) if self.kind == "qc" else 0

    @property
    def E(self) -> int:
        if self.kind == "qc":
            return int((self.shifts >= 0).sum()) * self.Z
        return int(self.col_idx.shape[0])


def qc_code(shifts, Z: int, name: str = "") -> Code:
    s = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32))
    if s.ndim != 2:
        raise ValueError("exponent matrix must be 2-D")
    if ((s < -1) | (s >= Z)).any():
        raise ValueError("shifts must lie in {-1, 0, ..., Z-1}")
    return Code("qc", n=s.shape[1] * Z, m=s.shape[0] * Z, Z=int(Z), shifts=s, name=name)


def csr_code(n: int, m: int, row_ptr, col_idx, name: str = "") -> Code:
    rp = np.ascontiguousarray(np.asarray(row_ptr, dtype=np.int32))
    ci = np.ascontiguousarray(np.asarray(col_idx, dtype=np.int32))
    if rp.shape != (m + 1,) or rp[0] != 0 or rp[-1] != ci.shape[0]:
        raise ValueError("bad row_ptr")
    return Code("csr", n=int(n), m=int(m), row_ptr=rp, col_idx=ci, name=name)


# --------------------------------------------------------------------------
# girth check used only to accept or redraw a random draw
# --------------------------------------------------------------------------

def _qc_adjacency(shifts: np.ndarray, Z: int):
    """Padded adjacency of the bipartite graph; node ids: VN v, CN n + c."""
    m_b, n_b = shifts.shape
    n, m = n_b * Z, m_b * Z
    vn = [[] for _ in range(n)]
    cn = [[] for _ in range(m)]
    for i in range(m_b):
        for j in range(n_b):
            a = int(shifts[i, j])
            if a < 0:
                continue
            for r in range(Z):
                c, v = i * Z + r, j * Z + (r + a) % Z
                cn[c].append(v)
                vn[v].append(c)
    N = n + m
    deg = np.array([len(x) for x in vn] + [len(x) for x in cn], dtype=np.int64)
    width = max(1, int(deg.max()))
    adj = np.full((N, width), -1, dtype=np.int64)
    for v in range(n):
        adj[v, : len(vn[v])] = [n + c for c in vn[v]]
    for c in range(m):
        adj[n + c, : len(cn[c])] = cn[c]
    return adj


def _shortest_cycle_through(adj: np.ndarray, s: int, limit: int) -> int:
    """Length of the shortest cycle through node s, or a value > limit if none <= limit."""
    N = adj.shape[0]
    dist = np.full(N, -1, dtype=np.int64)
    parent = np.full(N, -1, dtype=np.int64)
    dist[s] = 0
    frontier = np.array([s], dtype=np.int64)
    best = limit + 1
    d = 0
    while frontier.size and 2 * d + 1 < best:
        nb = adj[frontier]  # [F, W]
        src = np.repeat(frontier, nb.shape[1])
        nb = nb.reshape(-1)
        keep = (nb >= 0) & (nb != parent[src])
        src, nb = src[keep], nb[keep]
        seen = dist[nb] >= 0
        if seen.any():
            best = min(best, int((dist[src[seen]] + dist[nb[seen]] + 1).min()))
        new_src, new = src[~seen], nb[~seen]
        if new.size:
            uniq, first, counts = np.unique(new, return_index=True, return_counts=True)
            if (counts > 1).any():
                best = min(best, 2 * (d + 1))
            dist[uniq] = d + 1
            parent[uniq] = new_src[first]
            frontier = uniq
        else:
            frontier = new
        d += 1
    return best


def qc_girth_at_least(shifts: np.ndarray, Z: int, g: int) -> bool:
    """True iff every cycle of the QC Tanner graph has length >= g.

    By the circulant symmetry every cycle can be shifted to pass through a
    variable node (j, 0), so searching from those n_b nodes suffices.
    """
    adj = _qc_adjacency(shifts, Z)
    for j in range(shifts.shape[1]):
        if (shifts[:, j] >= 0).sum() == 0:
            continue
        if _shortest_cycle_through(adj, j * Z, g - 1) < g:
            return False
    return True


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------

def _closes_4cycle(E: np.ndarray, j: int, Z: int) -> bool:
    """Does column j close a 4-cycle with an earlier column?  Columns j, j'
    and rows i1, i2 (all blocks non-zero) form a 4-cycle iff the walk
    (i1,j) -> (i1,j') -> (i2,j') -> (i2,j) returns to its start modulo Z."""
    rows = np.flatnonzero(E[:, j] >= 0)
    for a in range(len(rows)):
        for b in range(a + 1, len(rows)):
            i1, i2 = rows[a], rows[b]
            prev = np.flatnonzero((E[i1, :j] >= 0) & (E[i2, :j] >= 0))
            if prev.size == 0:
                continue
            d = (E[i1, j] - E[i1, prev] + E[i2, prev] - E[i2, j]) % Z
            if (d == 0).any():
                return True
    return False


def draw_qc_columns(rng: np.random.Generator, m_b: int, n_b: int, Z: int, girth_min: int,
                    mask: Optional[np.ndarray] = None, max_tries: int = 20000, name: str = "") -> Code:
    """Column-greedy draw for larger bases: column j's shifts are drawn
    uniformly over [0, Z) and redrawn until the column closes no 4-cycle
    with columns 0..j-1; the finished matrix is accepted only if its girth
    (breadth-first search) is >= girth_min, else drawn again."""
    msk = np.ones((m_b, n_b), dtype=bool) if mask is None else np.asarray(mask, dtype=bool)
    for attempt in range(1, 101):
        E = np.full((m_b, n_b), -1, dtype=np.int64)
        ok = True
        for j in range(n_b):
            for _ in range(max_tries):
                E[:, j] = np.where(msk[:, j], rng.integers(0, Z, m_b), -1)
                if girth_min <= 4 or not _closes_4cycle(E, j, Z):
                    break
            else:
                ok = False
                break
        if ok and qc_girth_at_least(E.astype(np.int32), Z, girth_min):
            code = qc_code(E.astype(np.int32), Z, name=name)
            code.meta.update(attempts=attempt, girth_min=girth_min)
            return code
    raise RuntimeError(f"no {m_b}x{n_b} Z={Z} draw with girth >= {girth_min}")


def draw_qc(seed: int, m_b: int, n_b: int, Z: int, girth_min: int,
            mask: Optional[np.ndarray] = None, max_draws: int = 10000,
            rng: Optional[np.random.Generator] = None, name: str = "") -> Code:
    """Uniform shift draw over [0, Z), redrawn whole until girth >= girth_min."""
    rng = np.random.default_rng(seed) if rng is None else rng
    msk = np.ones((m_b, n_b), dtype=bool) if mask is None else np.asarray(mask, dtype=bool)
    for draw in range(1, max_draws + 1):
        E = rng.integers(0, Z, (m_b, n_b))
        E = np.where(msk, E, -1).astype(np.int32)
        if qc_girth_at_least(E, Z, girth_min):
            code = qc_code(E, Z, name=name)
            code.meta.update(seed=seed, draws=draw, girth_min=girth_min)
            return code
    raise RuntimeError(f"no draw with girth >= {girth_min} in {max_draws} draws")


def peg(seed: int, n: int, m: int, dv: int, dc: int, name: str = "") -> Code:
    """(dv, dc)-regular progressive-edge-growth graph; see the module docstring."""
    if n * dv != m * dc:
        raise ValueError("n*dv must equal m*dc for a regular graph")
    rng = np.random.default_rng(seed)
    deg_c = np.zeros(m, dtype=np.int64)
    vn_chk: list[list[int]] = [[] for _ in range(n)]
    chk_vn: list[list[int]] = [[] for _ in range(m)]

    def pick(cands: np.ndarray) -> int:
        d = deg_c[cands]
        ties = cands[d == d.min()]
        return int(ties[rng.integers(0, ties.size)]) if ties.size > 1 else int(ties[0])

    for v in range(n):
        for k in range(dv):
            eligible = deg_c < dc
            for c in vn_chk[v]:
                eligible[c] = False
            if not eligible.any():
                raise RuntimeError("PEG ran out of eligible checks")
            if k == 0:
                cands = np.flatnonzero(eligible)
            else:
                reached = np.zeros(m, dtype=bool)
                reached[vn_chk[v]] = True
                seen_v = {v}
                frontier = list(vn_chk[v])
                while True:
                    new_v = []
                    for c in frontier:
                        for u in chk_vn[c]:
                            if u not in seen_v:
                                seen_v.add(u)
                                new_v.append(u)
                    new_c = set()
                    for u in new_v:
                        for c in vn_chk[u]:
                            if not reached[c]:
                                new_c.add(c)
                    outside = eligible & ~reached
                    if not new_c:
                        cands = np.flatnonzero(outside)
                        break
                    nxt = reached.copy()
                    nxt[list(new_c)] = True
                    if not (eligible & ~nxt).any():
                        cands = np.flatnonzero(outside)
                        break
                    reached = nxt
                    frontier = list(new_c)
            c = pick(cands)
            deg_c[c] += 1
            vn_chk[v].append(c)
            chk_vn[c].append(v)
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum([len(x) for x in chk_vn])
    col_idx = np.concatenate([np.sort(np.array(x, dtype=np.int32)) for x in chk_vn])
    code = csr_code(n, m, row_ptr, col_idx, name=name)
    code.meta.update(seed=seed, dv=dv, dc=dc)
    return code


_BATCH_Z = (32, 64, 128, 256, 384)


def batch_codes(seeds=range(100, 132)) -> list[Code]:
    """Codes of the batching workload: 4 x n_b bases, n_b in [16, 32].

    Per seed: ``rng = default_rng(seed)``; n_b = rng.integers(16, 33); Z is
    drawn uniformly from those of (32, 64, 128, 256, 384) with Z >= 2 n_b
    (with 4 rows a girth-6 code needs distinct shift differences per row
    pair, so n_b <= Z at least); each column has weight 4 or 3 with equal
    probability, a weight-3 column gets its zero block in a row drawn
    uniformly; then ``draw_qc_columns`` with the same generator, girth >= 6.
    """
    out = []
    for seed in seeds:
        rng = np.random.default_rng(seed)
        n_b = int(rng.integers(16, 33))
        zs = [z for z in _BATCH_Z if z >= 2 * n_b]
        Z = int(zs[int(rng.integers(0, len(zs)))])
        mask = np.ones((4, n_b), dtype=bool)
        w3 = rng.integers(0, 2, n_b).astype(bool)
        rows = rng.integers(0, 4, n_b)
        for j in range(n_b):
            if w3[j]:
                mask[rows[j], j] = False
        code = draw_qc_columns(rng, 4, n_b, Z, 6, mask=mask, name=f"batch{seed}")
        code.meta.update(seed=seed)
        out.append(code)
    return out


def serving_codes(seed: int, count: int) -> list[Code]:
    """Codes of the serving stream: bases 3x6 .. 4x24, Z in [16, 512], n <= 10,000.

    Per code i: ``rng = default_rng((seed, i))``; m_b in {3, 4}; n_b in
    [2 m_b, 24]; Z drawn from powers of two and their 1.5x multiples in
    [16, 512] with 2 n_b <= Z and n_b * Z <= 10,000; full base (all blocks
    non-zero); ``draw_qc_columns``, girth >= 6.
    """
    zs = [16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512]
    out = []
    for i in range(count):
        rng = np.random.default_rng((seed, i))
        m_b = int(rng.integers(3, 5))
        n_b = int(rng.integers(2 * m_b, 25))
        ok = [z for z in zs if n_b * z <= 10000 and z >= 2 * n_b]
        Z = int(ok[int(rng.integers(0, len(ok)))])
        out.append(draw_qc_columns(rng, m_b, n_b, Z, 6, name=f"serve{seed}_{i}"))
    return out


# --------------------------------------------------------------------------
# named workloads: code + decoder + candidate rule
# --------------------------------------------------------------------------

WORKLOADS = {
    # 3x6 all-ones base, Z=16, seed 0, girth >= 6; int16 NMS, K=20, base +16, 10 steps
    "qc96": dict(code=lambda: draw_qc(0, 3, 6, 16, 6, name="qc96"),
                 K=20, base_llr=16, amp_steps=10, max_size=3, radius=4, cycle_len=0),
    # PEG (3,6) n=1008 seed 1; K=50, base +16, 12 steps
    "peg1008": dict(code=lambda: peg(1, 1008, 504, 3, 6, name="peg1008"),
                    K=50, base_llr=16, amp_steps=12, max_size=3, radius=4, cycle_len=0),
    # 3x6 all-ones base, Z=440, seed 2, girth >= 8; K=100, base +12, 10 steps
    "qc2640": dict(code=lambda: draw_qc(2, 3, 6, 440, 8, name="qc2640"),
                   K=100, base_llr=12, amp_steps=10, max_size=3, radius=4, cycle_len=8),
}

_CACHE: dict = {}


def workload(name: str) -> dict:
    """The named workload with its code built (cached per process)."""
    if name not in _CACHE:
        w = dict(WORKLOADS[name])
        w["code"] = w["code"]()
        w["name"] = name
        _CACHE[name] = w
    return _CACHE[name]
