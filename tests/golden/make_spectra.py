"""Writes the oracle's full-size trapping-set spectra that the GPU parity
tests compare against (``spectrum_*.npz`` beside this script).

Only the oracle (``oracle/``) computes anything here; the inputs come from
the seeded generators of ``synth/``.  The candidates are split into chunks
that worker processes (``spawn``) enumerate one at a time with the oracle as
it stands; the per-chunk lists of distinct trapping sets are merged by
canonical key (counts add, the threshold is the minimum), which is what one
oracle call over all candidates gives.

Workloads:
  qc2640 -- the 2640-node QC code, every canonical candidate (balls of size
            1..3 and the 8-cycle sets of size 4), K = 100, base 12, s = 10.
  peg1008_shard -- the 1008-node PEG code (K = 50, base 16, s = 12), the
            candidates that belong to representatives 0 .. R-1, R the
            smallest count with at least 200,000 candidates.  A candidate
            set belongs to its smallest member v whose Tanner ball holds
            every other member (general codes have no automorphism, so
            every variable node is a representative).

  code1_emd -- the EMD spectrum of Code 1 (Table V) up to 12-cycles: per
            cycle length 2l and EMD e, the oracle's class-weighted count
            (count2l; count2l / 2l cycles per circulant orbit), from the 20
            representatives (j, 0) (written to emd_code1_l6.txt).

  python tests/golden/make_spectra.py [qc2640|peg1008_shard|code1_emd ...] [--procs N]
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

SHARD_MIN = 200_000


def _params(w):
    return dict(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"], max_size=w["max_size"],
                cycle_len=w["cycle_len"])


def _work(args):
    name, rows = args
    w = synth.workload(name)
    g = oracle.Graph(w["code"])
    res = g.enumerate(rows, **_params(w))
    ts = [(t.key, t.a, t.b, t.orbit, int(t.elementary), t.count, t.thr) for t in res.ts_list]
    keys = [res.ts_list[i].key if i >= 0 else None for i in res.ts]
    return res.thr, res.decodes, res.iters, res.which, keys, ts


def owned_prefix(g, cands, min_count):
    """Candidates of representatives 0..R-1 (R smallest with >= min_count)."""
    balls = {}

    def ball(v):
        if v not in balls:
            balls[v] = set(g.ball4(v).tolist())
        return balls[v]

    def owner(row):
        S = [int(x) for x in row[1:1 + row[0]]]
        for v in sorted(S):
            if all(u == v or u in ball(v) for u in S):
                return v
        raise AssertionError(f"set {S} has no generating member")

    lo = cands[:, 1]  # the smallest member bounds the owner from below
    for R in range(1, g.n + 1):
        sel = np.flatnonzero(lo < R)
        own = np.array([owner(cands[i]) for i in sel])
        mine = sel[own < R]
        if len(mine) >= min_count:
            return R, cands[np.sort(mine)]
    raise AssertionError("code too small for the shard")


def spectrum(name, procs):
    t0 = time.time()
    base = "peg1008" if name == "peg1008_shard" else name
    w = synth.workload(base)
    g = oracle.Graph(w["code"])
    cands = g.candidates(w["max_size"], w["cycle_len"])
    meta = dict(workload=base, **_params(w), n_cand_code=int(len(cands)))
    if name == "peg1008_shard":
        R, cands = owned_prefix(g, cands, SHARD_MIN)
        meta["representatives"] = R
    n = len(cands)
    chunks = np.array_split(np.arange(n), max(1, min(n, procs * 16)))
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_work, [(base, cands[c]) for c in chunks], chunksize=1)
    thr = np.concatenate([p[0] for p in parts]).astype(np.int32)
    dec = np.concatenate([p[1] for p in parts]).astype(np.int32)
    it = np.concatenate([p[2] for p in parts]).astype(np.int32)
    which = np.concatenate([p[3] for p in parts]).astype(np.int32)
    keys = [k for p in parts for k in p[4]]
    merged = {}
    for p in parts:
        for key, a, b, orbit, elem, count, t in p[5]:
            if key in merged:
                m = merged[key]
                assert (m[0], m[1], m[2], m[3]) == (a, b, orbit, elem)
                m[4] += count
                m[5] = min(m[5], t)
            else:
                merged[key] = [a, b, orbit, elem, count, t]
    order = sorted(merged, key=lambda k: (merged[k][0], merged[k][1], k))
    index = {k: i for i, k in enumerate(order)}
    ts = np.array([index[k] if k is not None else -1 for k in keys], dtype=np.int32)
    tab = np.array([merged[k] for k in order], dtype=np.int32).reshape(-1, 6)
    key_off = np.zeros(len(order) + 1, dtype=np.int64)
    key_off[1:] = np.cumsum([len(k) for k in order])
    flat = np.array([x for k in order for x in k], dtype=np.int32)
    meta.update(n_cand=int(n), n_ts=len(order), core_seconds=None, wall_s=round(time.time() - t0, 1),
                procs=procs)
    out = os.path.join(HERE, f"spectrum_{name}.npz")
    np.savez_compressed(out, cands=cands.astype(np.int32), thr=thr, decodes=dec, iters=it, which=which, ts=ts,
                        ts_a=tab[:, 0], ts_b=tab[:, 1], ts_orbit=tab[:, 2], ts_elem=tab[:, 3], ts_count=tab[:, 4],
                        ts_thr=tab[:, 5], key_off=key_off, keys=flat, meta=np.array(json.dumps(meta)))
    print(f"{name}: {n} candidates, {len(order)} trapping sets, {time.time() - t0:.0f} s -> {out}", flush=True)


def _walks_job(args):
    code, v, lmax = args
    return oracle.Graph(code).cycle_walks(v, lmax, emd=True)


def code1_emd(procs, lmax=6):
    t0 = time.time()
    rows, Z = [], None
    with open(os.path.join(HERE, "code1_table5.txt")) as f:
        for line in f:
            tok = line.split("#", 1)[0].split()
            if tok and tok[0] == "Z":
                Z = int(tok[1])
            elif tok and tok[0][0] in "-0123456789":
                rows.append([int(x) for x in tok])
    code = synth.qc_code(np.array(rows, dtype=np.int32), Z)
    with mp.get_context("spawn").Pool(procs) as pool:
        parts = pool.map(_walks_job, [(code, j * Z, lmax) for j in range(len(rows[0]))], chunksize=1)
    hist = sum(p[1] for p in parts)
    walks = sum(p[0] for p in parts)
    out = os.path.join(HERE, "emd_code1_l6.txt")
    with open(out, "w") as f:
        f.write("# The oracle's EMD spectrum of Code 1 (Table V), written by make_spectra.py code1_emd:\n"
                "# closed exponent chains (Prop. 1) of l = 2..6 variable nodes from the representatives (j, 0);\n"
                "# count2l / (2 l) is the number of cycles of length 2l and EMD e per circulant orbit.\n"
                "# l emd count2l   (and: walks l total)\n")
        for l in range(2, lmax + 1):
            f.write(f"walks {l} {int(walks[l])}\n")
            for e in np.flatnonzero(hist[l]):
                f.write(f"{l} {int(e)} {int(hist[l, e])}\n")
    print(f"code1_emd: {time.time() - t0:.0f} s -> {out}", flush=True)


def main():
    names = [a for a in sys.argv[1:] if not a.startswith("--") and not a.isdigit()] or \
        ["qc2640", "peg1008_shard", "code1_emd"]
    procs = os.cpu_count() or 1
    if "--procs" in sys.argv:
        procs = int(sys.argv[sys.argv.index("--procs") + 1])
    for name in names:
        if name == "code1_emd":
            code1_emd(procs)
        else:
            spectrum(name, procs)


if __name__ == "__main__":
    main()
