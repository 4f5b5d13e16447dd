#!/usr/bin/env python
"""Benchmark: impulse-decode edge-updates/s of the trapping-set enumeration.

One step = one enumerate_ts() call on the workload: candidate generation and
canonical dedupe, impulse decodes with amplitude bisection, sieving,
classification, canonical form and dedupe of the trapping sets -- the whole
hot path -- over every canonical candidate of the code.  Inputs (the code's
device tables) are resident when the timed region starts; L2 is flushed
(a 256 MB write) before every timed step, outside its CUDA-event bracket.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batch32 [--tune]   # 32 codes, one graph-replayed batch
  python bench.py --workload serve [--jobs N --load F]   # Poisson job stream, p50/p99
  python bench.py --workload isfer [--samples N]          # importance-sampling FER job

The batch32 workload enumerates the 32 QC codes of uneven sizes (4 x 16 to
4 x 32 bases, Z 64 to 384) together: per-code candidate kernels and sieves,
one multi-code persistent decode launch, the whole step captured once in a
CUDA graph and replayed; the same codes run one enumerate_ts() at a time are
timed beside it ("serial").

At one GPU the default run also measures, after the headline, the other
workloads of the library with a few steps each and reports them as extra
keys of the one JSON line: the batch of 32 codes (tuned tiles, against one
enumerate_ts() per code), the serving stream (p50/p99 against the plain
one-job-at-a-time method, results compared), and the importance-sampling
job (--no-extras skips them).

Rooflines: the decoders are bound by integer issue and shared-memory
bandwidth; measure_peaks() measures both per SM clock on the device, and the
peak is taken at the SM clock sampled during the timed region.  The
two-codeword kernels do two edge updates per 16-bit-pair lane operation.

Multi-GPU (torchrun): every rank enumerates its own code of the same shape
(rank r uses seed offset r: independent problems, weak scaling); no
collective on the data path, a barrier and max-over-ranks time only.
--impl reference times the CPU oracle, as it stands, on a bounded sample of
the same workload each step, over all host cores (one process per core).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from paper_2208_05795_gb300.shard import exchange, reduce_time_and_work, shard_bounds, ts_records  # noqa: E402

# integer operations the min-sum edge update needs at minimum: |q|, two
# compare-selects for min1/min2, argmin select, sign xor, output select,
# x3, >>2, sign apply, the add of the variable-node sum, the subtract of
# P - r and the two-sided clamp (counted as one)
ALG_OPS_PER_EDGE = 12
# shared-memory bytes an edge update needs at minimum: write and read one
# 16-bit check-to-variable message (posterior and variable-to-check message
# are recomputable)
ALG_SMEM_BYTES_PER_EDGE = 4
# DRAM bytes (read + write) an ncu capture measured for the PEG decode launch over its first
# 40,000 candidates; None until captured for the kernel as it stands
PAIR_KERNEL_DRAM_BYTES_40K = 726528.0
SM_MAX_MHZ = 2070.0
try:  # the maximum SM clock measured on this machine, when the measurement file is present
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        SM_MAX_MHZ = float(json.load(_f).get("sm_max_mhz", SM_MAX_MHZ))
except (OSError, ValueError):
    pass


def alu_roofline(eu_per_launch, ms_launch, pk, sm_mhz, packed=True, traffic=None, note=""):
    """Roofline of a min-sum decode launch in edge updates per second:
    min(integer lane-ops/s x values per lane-op / 12, shared-memory B/s / 4),
    from the measured per-clock rates at the sampled SM clock."""
    mhz = sm_mhz or SM_MAX_MHZ
    clk = mhz * 1e6 * pk["num_sms"]
    per_op = 2 if packed else 1
    lane = pk["u16x2_ops_per_clk_sm"] if packed else pk["int32_ops_per_clk_sm"]
    int_bound = lane * clk * per_op / ALG_OPS_PER_EDGE
    smem_bound = pk["smem_bytes_per_clk_sm"] * clk / ALG_SMEM_BYTES_PER_EDGE
    peak = min(int_bound, smem_bound)
    achieved = eu_per_launch / (ms_launch / 1e3)
    unpacked = pk["int32_ops_per_clk_sm"] * clk / ALG_OPS_PER_EDGE
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "edge-updates/s", "frac": achieved / peak,
            "traffic": traffic,
            "terms": {"int_bound": int_bound, "smem_bound": smem_bound, "sm_mhz": mhz, "num_sms": pk["num_sms"],
                      "int32_ops_per_clk_sm": pk["int32_ops_per_clk_sm"],
                      "u16x2_ops_per_clk_sm": pk["u16x2_ops_per_clk_sm"],
                      "smem_bytes_per_clk_sm": pk["smem_bytes_per_clk_sm"], "ops_per_edge": ALG_OPS_PER_EDGE,
                      "values_per_lane_op": per_op, "smem_bytes_per_edge": ALG_SMEM_BYTES_PER_EDGE,
                      "achieved_int_ops_per_s": ALG_OPS_PER_EDGE * achieved,
                      "frac_of_unpacked_int32": achieved / unpacked},
            "note": note or "peaks measured by measure_peaks() per SM clock, at the sampled median SM clock"}


# the extra workloads, also runnable on their own (one JSON line each):
# name -> (metric, unit, key of the value in the extra's summary)
EXTRA_WORKLOADS = {
    "list2640": ("ordered-list distinct trapping sets/s", "trapping sets/s", "distinct_ts_per_s"),
    "budget_code1": ("iteration-budget speed-up over K for all", "x", "speedup"),
    "lnms_code1": ("layered-decoder frames/s", "frames/s", "frames_per_s"),
    "emd_code1": ("EMD spectrum search time", "ms", "ms"),
    "spa_peg": ("sum-product edge-updates/s", "edge-updates/s", "edge_updates_per_s"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="peg1008",
                    choices=sorted(synth.WORKLOADS) + ["batch32", "serve", "isfer"] + sorted(EXTRA_WORKLOADS))
    ap.add_argument("--samples", type=int, default=1_000_000, help="isfer: samples per step")
    ap.add_argument("--no-graph", action="store_true", help="batch32: launch each step eagerly instead of "
                                                             "replaying the captured graph")
    ap.add_argument("--batch-seeds", default="", help="batch32: comma-separated code seeds instead of 100..131 "
                                                      "(a bounded case for profiling)")
    ap.add_argument("--jobs", type=int, default=120, help="serve: jobs in the Poisson stream")
    ap.add_argument("--load", type=float, default=0.8, help="serve: offered load (fraction of the plain method's "
                                                             "throughput)")
    ap.add_argument("--tune", action="store_true", help="batch32: pick each code's tile with tune_tile()")
    ap.add_argument("--decoder", default="nms16", choices=["nms16", "nms8", "spa"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cand-limit", type=int, default=-1,
                    help="decode only the first N canonical candidates (profiling a bounded case)")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only (no extra workloads)")
    ap.add_argument("--procs", type=int, default=0, help="oracle processes (0 = every host core)")
    ap.add_argument("--split", action="store_true",
                    help="several ranks: split one code's canonical candidate list into contiguous ranges "
                         "(strong scaling) and merge the per-range trapping sets in one exchange step, "
                         "instead of one independent code per rank")
    return ap.parse_args()


def rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def workload_for(name, rank):
    if name == "batch32":  # the reference arm samples the first code of the batch
        return dict(code=synth.batch_codes([100 + 32 * rank])[0], **BATCH)
    if name in ("serve", "isfer"):  # the reference arm samples the largest code of the stream
        return dict(code=synth.serving_codes(2026, 8)[4], **SERVE_ENUM)
    w = dict(synth.workload(name))
    if rank:
        if name == "peg1008":
            w["code"] = synth.peg(1 + rank, 1008, 504, 3, 6, name=f"peg1008_s{1 + rank}")
        elif name == "qc96":
            w["code"] = synth.draw_qc(rank, 3, 6, 16, 6)
        else:
            w["code"] = synth.draw_qc(2 + rank, 3, 6, 440, 8)
    return w


def params_of(w, decoder):
    return dict(decoder=decoder, K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"],
                max_size=w["max_size"], cycle_len=w["cycle_len"])


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        busy = [r for r in rows if r[4].isdigit() and int(r[4]) >= 50] or rows
        sm = [float(r[1]) for r in busy if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in busy for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": reasons, "samples": len(busy)}


def _oracle_chunk(job):
    """One worker's share of an oracle timing: (iterations, seconds)."""
    import oracle
    code, rows, p, od = job
    g = oracle.Graph(code)
    t0 = time.perf_counter()
    res = g.enumerate(rows, decoder=od, **p)
    return int(res.iters.sum()), time.perf_counter() - t0


class OraclePool:
    """The oracle on every host core: one spawned process per core (spawned,
    so that no worker inherits a CUDA context)."""

    def __init__(self, procs=0):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def run(self, code, rows, p, od):
        """Wall seconds and summed iterations of enumerating `rows`, split over
        the processes."""
        chunks = [c for c in np.array_split(rows, self.procs * 4) if len(c)]
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_chunk, [(code, c, p, od) for c in chunks], chunksize=1)
        return time.perf_counter() - t0, sum(o[0] for o in out)

    def close(self):
        self.pool.close()
        self.pool.join()


def _oracle_args(w, decoder):
    p = params_of(w, decoder)
    p.pop("decoder")
    if decoder == "nms8":
        p["sat"] = 127
    return p, ("spa" if decoder == "spa" else "nms")


def cpu_baseline(w, decoder, seconds, rng_seed=0, procs=0):
    """The oracle, as it stands, on bounded random samples of the workload's
    canonical candidates: single-threaded, then over every host core;
    edge-updates/s."""
    import oracle
    g = oracle.Graph(w["code"])
    cands = g.candidates(w["max_size"], w["cycle_len"])
    rng = np.random.default_rng(rng_seed)
    p, od = _oracle_args(w, decoder)
    n, it, el, ncand = 4, 0, 0.0, 0
    while el < seconds / 2:
        pick = rng.choice(len(cands), min(n, len(cands)), replace=False)
        t0 = time.perf_counter()
        res = g.enumerate(cands[np.sort(pick)], decoder=od, **p)
        el += time.perf_counter() - t0
        it += int(res.iters.sum())
        ncand += len(pick)
        n = min(len(cands), n * 2)
    single = {"value": it * g.E / el, "cores": 1,
              "sample": f"{ncand} random canonical candidates of {len(cands)} (seeded), {el:.1f} s"}
    rate1 = ncand / el
    pool = OraclePool(procs)
    try:
        pool.run(w["code"], cands[:pool.procs], p, od)  # start the workers
        want = int(rate1 * pool.procs * seconds / 2) + pool.procs
        pick = np.sort(rng.choice(len(cands), min(want, len(cands)), replace=False))
        wall, it_all = pool.run(w["code"], cands[pick], p, od)
    finally:
        pool.close()
    return {"value": it_all * g.E / wall, "unit": "edge-updates/s", "cores": pool.procs, "kind": "oracle",
            "nproc": os.cpu_count(),
            "sample": f"{len(pick)} random canonical candidates of {len(cands)} (seeded), {wall:.1f} s wall over "
                      f"{pool.procs} processes",
            "single_thread": single}, rate1


def run_reference(args):
    rank, world, _ = rank_world()
    if rank != 0:
        return
    w = workload_for(args.workload, 0)
    times, eus = [], []
    import oracle
    g = oracle.Graph(w["code"])
    cands = g.candidates(w["max_size"], w["cycle_len"])
    p, od = _oracle_args(w, args.decoder)
    rng = np.random.default_rng(1)
    pool = OraclePool(args.procs)
    try:
        # per step about 3 s of the pool's time, from a calibration sample
        pool.run(w["code"], cands[:pool.procs], p, od)  # start the workers
        cal = np.sort(rng.choice(len(cands), min(len(cands), 16 * pool.procs), replace=False))
        wall, _ = pool.run(w["code"], cands[cal], p, od)
        per_step = int(min(len(cands), max(pool.procs, len(cal) * 3.0 / max(wall, 1e-3))))
        for s in range(args.warmup + args.steps):
            pick = np.sort(rng.choice(len(cands), per_step, replace=False))
            dt, it = pool.run(w["code"], cands[pick], p, od)
            if s >= args.warmup:
                times.append(dt)
                eus.append(it * g.E)
    finally:
        pool.close()
    value = sum(eus) / sum(times)
    line = {"impl": "reference", "metric": "impulse-decode edge-updates/s", "value": value,
            "unit": "edge-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.decoder == "spa" else "int16", "data": "synthetic",
            "config": {"workload": args.workload, "decoder": args.decoder,
                       "sample_per_step": per_step, "n_cand": int(len(cands))},
            "cpu_baseline": {"value": value, "unit": "edge-updates/s", "cores": pool.procs, "kind": "oracle",
                             "nproc": os.cpu_count(),
                             "sample": f"{per_step} random canonical candidates per step over {pool.procs} "
                                       f"processes"},
            "e2e": {"value": value, "unit": "edge-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2208_05795_gb300 as tsx
    from paper_2208_05795_gb300 import build as tsx_build

    rank, world, local = rank_world()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    tsx_build.build()
    pk = tsx.measure_peaks()
    split = args.split and world > 1
    w = workload_for(args.workload, 0 if split else rank)
    params = params_of(w, args.decoder)
    if args.decoder == "nms8":
        params["sat"] = 127
    if args.cand_limit >= 0:
        params["cand_end"] = args.cand_limit
    stream = torch.cuda.Stream()
    code = tsx.load_code(w["code"], stream=stream)
    shard_range, shard_n_total = None, 0
    if split:
        # this rank's contiguous range of the one code's canonical list
        n_total = tsx.ts_list_stats(tsx.enumerate_ts(code, stream=stream, **dict(params, cand_end=0)))["n_cand_total"]
        if args.cand_limit >= 0:
            n_total = min(n_total, args.cand_limit)
        shard_range, shard_n_total = shard_bounds(n_total, rank, world), n_total
        params.update(cand_begin=shard_range[0], cand_end=shard_range[1])
    info = code.info
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    has_cycles = w["cycle_len"] // 2 > w["max_size"]
    # candidates (count, scan, write; again for cycle sets), decode, sieve, compaction (2)
    launches_per_step = 3 + (3 if has_cycles else 0) + 1 + 1 + 2

    def step():
        return tsx.enumerate_ts(code, stream=stream, **params)

    for _ in range(args.warmup):
        tsx.ts_list_stats(step())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times, eu, dec, nts, ms_dec, ms_cand = [], 0, 0, 0, [], []
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lst = step()
            e1.record(stream)
            s = tsx.ts_list_stats(lst)
            times.append(e0.elapsed_time(e1))
            eu += s["edge_updates"]
            dec += s["decodes"]
            nts = s["n_ts"]
            ms_dec.append(s["ms_decode"])
            ms_cand.append(s["ms_candidates"])
            del lst
        torch.cuda.synchronize()
    clocks = clk.summary()
    total_ms = sum(times)
    if dist:
        total_ms, (eu_all, dec_all) = reduce_time_and_work(total_ms, [eu, dec], device="cuda")
    else:
        eu_all, dec_all = float(eu), float(dec)
    value = eu_all / (total_ms / 1e3)

    # end to end through the public API with host buffers
    e2e = None
    if args.e2e_steps > 0:
        wall, eu2, h2d, d2h = 0.0, 0, 0, 0
        desc_bytes = (w["code"].shifts.nbytes if w["code"].kind == "qc"
                      else w["code"].row_ptr.nbytes + w["code"].col_idx.nbytes)
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c2 = tsx.load_code(w["code"], stream=stream)
            v = tsx.ts_list_view(tsx.enumerate_ts(c2, stream=stream, **params), keys=False)
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            eu2 += v["stats"]["edge_updates"]
            n_rep = c2.info["n_rep"]
            h2d = desc_bytes + 8 * (n_rep + 1)
            d2h = sum(v[k].nbytes for k in ("cand_vars", "cand_thr", "cand_thr_f", "cand_ts", "cand_flags",
                                            "cand_decodes", "cand_iters", "a", "b", "orbit", "count", "thr",
                                            "flags", "thr_f", "key_vars", "key_off"))
            del c2
        e2e = {"value": eu2 / wall, "unit": "edge-updates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    split_info = None
    if split:
        # the one exchange step: every range's (key -> record) map, merged by key on every rank
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        merged = exchange(ts_records(tsx.ts_list_view(step())))
        split_info = {"ranks": world, "cand_range_rank0": list(shard_range), "n_ts_merged": len(merged),
                      "ms_view_and_exchange": 1e3 * (time.perf_counter() - t0)}
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    avg_dec_ms = sum(ms_dec) / len(ms_dec)
    # DRAM bytes (read + write) of one decode launch, from an ncu capture of this kernel on the PEG
    # workload's first 40,000 candidates (profiles/pair_kernel_peg1008_40k.md), scaled to the launch's
    # candidates (candidate sets in, records out: both proportional to the candidates)
    traffic = None
    if args.workload == "peg1008" and args.decoder == "nms16" and PAIR_KERNEL_DRAM_BYTES_40K:
        traffic = PAIR_KERNEL_DRAM_BYTES_40K / 40000 * float(s["n_cand"])

    eu_per_step = eu / args.steps
    roof = (alu_roofline(eu_per_step, avg_dec_ms, pk, clocks.get("sm_mhz"), packed=args.decoder != "spa",
                         traffic=traffic) if args.decoder != "spa" else None)
    cpu = cpu_baseline(w, args.decoder, args.cpu_seconds, procs=args.procs)[0] if args.cpu_seconds > 0 else None
    extras = None
    if world == 1 and not args.no_extras:
        extras = run_extras(args, tsx, pk)
    line = {
        "metric": "impulse-decode edge-updates/s",
        "value": value,
        "unit": "edge-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "strong" if split else "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.decoder == "spa" else ("int8" if args.decoder == "nms8" else "int16"),
        "data": "synthetic",
        "config": {"workload": args.workload + (f"[:{args.cand_limit}]" if args.cand_limit >= 0 else ""),
                   "decoder": args.decoder, "n": info["n"], "m": info["m"],
                   "E": info["E"], "girth": info["girth"], "K": w["K"], "amp_steps": w["amp_steps"],
                   "base_llr": w["base_llr"], "n_cand": int(shard_n_total if split else s["n_cand"]),
                   "parallelism": f"split{world}" if split else f"replicas{world}",
                   "l2": "flushed before each step (256 MB write)"},
        "decodes_per_s": dec_all / (total_ms / 1e3),
        "distinct_ts_per_s": (split_info["n_ts_merged"] if split else nts * world) / (total_ms / args.steps / 1e3),
        "n_ts": nts,
        "ms_decode_kernel": avg_dec_ms,
        "ms_candidates": sum(ms_cand) / len(ms_cand),
        "roofline": roof,
        "measured_peaks": pk,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if split_info:
        line["split"] = split_info
    if extras:
        line["extra"] = extras
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


BATCH = dict(K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)


def run_batch(args, pk=None):
    import torch
    import paper_2208_05795_gb300 as tsx
    from paper_2208_05795_gb300 import build as tsx_build

    rank, world, local = rank_world()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    tsx_build.build()
    # rank r takes seeds 100 + 32 r .. 131 + 32 r: independent batches of the same shape
    seeds = ([int(x) for x in args.batch_seeds.split(",")] if args.batch_seeds
             else list(range(100 + 32 * rank, 132 + 32 * rank)))
    codes = synth.batch_codes(seeds)
    stream = torch.cuda.Stream()
    handles = [tsx.load_code(c, stream=stream) for c in codes]
    params = dict(BATCH, decoder=args.decoder)
    if args.decoder == "nms8":
        params["sat"] = 127
    base = tsx.make_params(**params)
    plist = [tsx.tune_tile(h, base, stream=stream)[0] if args.tune else base for h in handles]
    if args.tune and len({p.decoder for p in plist}) > 1:
        plist = [p if p.decoder == base.decoder else tsx.make_params(**dict(params, warps_per_cta=p.warps_per_cta))
                 for p in plist]
    batch = tsx.batch_create(handles, plist, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        tsx.batch_run(batch, stream=stream)
    stream.synchronize()
    if args.no_graph:  # eager launches (for a profiler that does not follow stream capture)
        def replay():
            tsx.batch_run(batch, stream=stream)
    else:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            tsx.batch_run(batch, stream=stream)
        replay = graph.replay
    for _ in range(args.warmup):
        replay()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times = []
    with Clocks(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                replay()
                e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
    clocks = clk.summary()
    s = tsx.batch_stats(batch)
    total_ms = sum(times)
    eu, dec, nts = float(s["edge_updates"]) * args.steps, float(s["decodes"]) * args.steps, s["n_ts"]
    if dist:
        total_ms, (eu, dec) = reduce_time_and_work(total_ms, [eu, dec], device="cuda")
    value = eu / (total_ms / 1e3)

    # the same codes one enumerate_ts() at a time (eager, per-code launches)
    serial_ms = []
    for _ in range(max(1, min(2, args.steps))):
        with torch.cuda.stream(stream):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lists = [tsx.enumerate_ts(h, p, stream=stream) for h, p in zip(handles, plist)]
            e1.record(stream)
        e1.synchronize()
        serial_ms.append(e0.elapsed_time(e1))
        del lists

    # end to end: load the 32 codes from host arrays, create, run, read back every result
    e2e = None
    if args.e2e_steps > 0:
        wall, eu2, h2d, d2h = 0.0, 0, 0, 0
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hs = [tsx.load_code(c, stream=stream) for c in codes]
            b2 = tsx.batch_create(hs, plist, stream=stream)
            tsx.batch_run(b2, stream=stream)
            views = [tsx.batch_view(b2, i, keys=False) for i in range(len(hs))]
            wall += time.perf_counter() - t0
            eu2 += sum(v["stats"]["edge_updates"] for v in views)
            h2d = sum(c.shifts.nbytes for c in codes)
            d2h = sum(sum(v[k].nbytes for k in ("cand_vars", "cand_thr", "cand_thr_f", "cand_ts", "cand_flags",
                                                "cand_decodes", "cand_iters", "a", "b", "orbit", "count", "thr",
                                                "flags", "thr_f", "key_vars", "key_off"))
                      for v in views)
            del b2, hs
        e2e = {"value": eu2 / wall, "unit": "edge-updates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return None
    if pk is None:
        pk = tsx.measure_peaks()
    ms_step = total_ms / args.steps
    line = {
        "metric": "impulse-decode edge-updates/s",
        "value": value,
        "unit": "edge-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int8" if args.decoder == "nms8" else "int16",
        "data": "synthetic",
        "config": {"workload": "batch32" + (f"[{args.batch_seeds}]" if args.batch_seeds else ""),
                   "codes": len(codes), "n_cand": int(s["n_cand"]),
                   "n_range": [min(c.n for c in codes), max(c.n for c in codes)], "decoder": args.decoder,
                   **BATCH, "tuned": bool(args.tune), "tiles": sorted({p.warps_per_cta for p in plist}),
                   "multi_code_launch": batch.multi_launch, "cuda_graph": not args.no_graph,
                   "parallelism": f"replicas{world}", "l2": "flushed before each step (256 MB write)"},
        "decodes_per_s": dec / (total_ms / 1e3),
        "n_ts": int(nts),
        "serial_ms_per_step": statistics.median(serial_ms),
        "batch_speedup_vs_serial": statistics.median(serial_ms) / ms_step,
        "roofline": alu_roofline(float(s["edge_updates"]), ms_step, pk, clocks.get("sm_mhz"),
                                 note="whole step (candidates, decode, sieve) against the decoders' bound"),
        "cpu_baseline": None,
        "e2e": e2e,
        # per code: candidates (3), sieve, compaction (2); plus the decode launches of the batch
        "gpu_launches": (len(codes) * 6 + batch.decode_launches) * args.steps,
        "clocks": clocks,
    }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


SERVE_ENUM = dict(K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)


def serve_jobs(n_jobs, seed=2026):
    """The serving stream's jobs (arrival times are drawn later from the
    offered load): 8 resident QC codes (bases 3x6 .. 4x24, Z 16 .. 512,
    n <= 10,000); 3 in 4 jobs enumerate 1K .. 100K candidates (log-uniform)
    of a code, the others run 10^6 importance samples toward a trapping set
    of a code found beforehand, at Eb/N0 uniform in [3, 5] dB."""
    rng = np.random.default_rng(seed)
    codes = synth.serving_codes(seed, 8)
    jobs = []
    for j in range(n_jobs):
        c = int(rng.integers(0, len(codes)))
        if rng.random() < 0.75:
            ncand = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
            jobs.append(("enum", c, dict(SERVE_ENUM, cand_end=ncand)))
        else:
            jobs.append(("is", c, dict(ebn0_db=float(rng.uniform(3.0, 5.0)), mu=1.0, n_samples=1_000_000,
                                        job_key=1000 + j)))
    return codes, jobs


def run_serve(args):
    import torch
    import paper_2208_05795_gb300 as tsx
    from paper_2208_05795_gb300 import build as tsx_build

    rank, world, local = rank_world()
    torch.cuda.set_device(local)
    if world > 1 and rank != 0:
        return None  # the serving stream runs on one GPU: replicas only
    tsx_build.build()
    codes, jobs = serve_jobs(args.jobs)
    handles = [tsx.load_code(c) for c in codes]
    # a trapping set per code for the importance-sampling jobs: the lowest
    # threshold among the first 2000 candidates' sets
    ts_of = []
    for h in handles:
        v = tsx.ts_list_view(tsx.enumerate_ts(h, **dict(SERVE_ENUM, cand_end=2000)))
        thr = np.where(v["thr"] >= 0, v["thr"], 1 << 30)
        ts_of.append(v["keys"][int(np.argmin(thr))] if len(thr) else (0,))

    def submit(srv, job):
        kind, c, p = job
        if kind == "enum":
            return srv.submit_enumerate(handles[c], **p)
        return srv.submit_is_fer(handles[c], ts_of[c], **p)

    def stream(srv, arrivals):
        ids = []
        t0 = time.perf_counter()
        for job, t in zip(jobs, arrivals):
            d = t - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            ids.append(submit(srv, job))
        srv.drain()
        res = [srv.wait(i) for i in ids]
        st = srv.stats()
        for i in ids:
            srv.release(i)
        return res, st

    # warm-up, then the plain method's throughput with every job queued at once
    with tsx.Server(serial=1) as srv:
        for job in jobs[:3]:
            srv.wait(submit(srv, job))
        srv.reset_stats()
        _, cal = stream(srv, [0.0] * len(jobs))
    mean_service_s = cal["makespan_ms"] / 1e3 / len(jobs)
    rate = args.load / mean_service_s
    arrivals = np.cumsum(np.random.default_rng(7).exponential(1.0 / rate, len(jobs)))
    arrivals -= arrivals[0]
    out = {}
    for mode, kw in (("plain", dict(serial=1)), ("served", dict(max_jobs=8))):
        with Clocks(local) as clk:
            with tsx.Server(**kw) as srv:
                res, st = stream(srv, list(arrivals))
        out[mode] = (res, st, clk.summary())
    rp, sp, _ = out["plain"]
    rs, ss, clocks = out["served"]
    launches = served_launches(jobs, rs)
    same = all(a["status"] == b["status"] == 0 and
               (a["enum_stats"]["n_ts"], a["enum_stats"]["decodes"], a["is_result"]["sum_w"],
                a["is_result"]["n_fail"]) ==
               (b["enum_stats"]["n_ts"], b["enum_stats"]["decodes"], b["is_result"]["sum_w"],
                b["is_result"]["n_fail"]) for a, b in zip(rp, rs))
    n_enum = sum(1 for j in jobs if j[0] == "enum")
    line = {
        "metric": "serving job latency p99",
        "value": ss["p99_ms"],
        "unit": "ms",
        "n_gpus": 1,
        "steps": len(jobs),
        "warmup": 3,
        "ms_per_step": ss["mean_ms"],
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int16",
        "data": "synthetic",
        "config": {"workload": "serve", "jobs": len(jobs), "enumeration_jobs": n_enum,
                   "is_jobs": len(jobs) - n_enum, "codes": len(codes),
                   "n_range": [min(c.n for c in codes), max(c.n for c in codes)],
                   "offered_load": args.load, "arrival_rate_per_s": rate,
                   "mean_service_ms_plain": mean_service_s * 1e3, "max_jobs": 8,
                   "l2": "inputs resident; not flushed (a stream of jobs)"},
        "p50_ms": ss["p50_ms"], "p90_ms": ss["p90_ms"], "p99_ms": ss["p99_ms"], "mean_ms": ss["mean_ms"],
        "plain": {"p50_ms": sp["p50_ms"], "p90_ms": sp["p90_ms"], "p99_ms": sp["p99_ms"], "mean_ms": sp["mean_ms"],
                  "edge_updates_per_s": sp["edge_updates_per_s"], "makespan_ms": sp["makespan_ms"]},
        "edge_updates_per_s": ss["edge_updates_per_s"],
        "makespan_ms": ss["makespan_ms"],
        "max_concurrent_jobs": ss["max_concurrent"],
        "hbm_peak_bytes": ss["hbm_peak_bytes"],
        "results_identical_to_plain": bool(same),
        "roofline": None,
        "cpu_baseline": None,
        "e2e": {"value": ss["p99_ms"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "latency is measured from submit (host) to results copied to host memory"},
        "gpu_launches": launches,
        "gpu_launches_note": "served mode, counted from each job's candidates or samples and the server's "
                             "chunk sizes (candidate bound taken as the canonical count: a lower bound)",
        "clocks": clocks,
    }
    return line


def served_launches(jobs, results, chunk_candidates=16384, chunk_samples=32768):
    """Kernel launches of the served stream: an enumeration job runs the
    candidate kernels (count, scan, write), one decode launch per chunk of
    candidates, the sieve and two compaction kernels; an importance-sampling
    job one sampling launch per chunk of samples and two reductions."""
    n = 0
    for (kind, _, p), r in zip(jobs, results):
        if kind == "enum":
            cands = max(1, int(r["enum_stats"]["n_cand"]))
            n += 3 + -(-cands // chunk_candidates) + 1 + 2
        else:
            n += -(-int(p["n_samples"]) // chunk_samples) + 2
    return n


def isfer_setup(tsx, stream=None):
    """The importance-sampling workload: the largest serving code (n = 8,832,
    4 x 23 base, Z = 384), biased toward the lowest-threshold trapping set
    among its first 2,000 candidates, at Eb/N0 = 4 dB, mu = 1."""
    code = synth.serving_codes(2026, 8)[4]
    h = tsx.load_code(code, stream=stream)
    v = tsx.ts_list_view(tsx.enumerate_ts(h, stream=stream, **dict(SERVE_ENUM, cand_end=2000)))
    thr = np.where(v["thr"] >= 0, v["thr"], 1 << 30)
    return code, h, v["keys"][int(np.argmin(thr))]


def run_isfer(args, pk=None):
    import torch
    import paper_2208_05795_gb300 as tsx
    from paper_2208_05795_gb300 import build as tsx_build

    rank, world, local = rank_world()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tsx_build.build()
    stream = torch.cuda.Stream()
    code, h, ts = isfer_setup(tsx, stream)
    kw = dict(ebn0_db=4.0, mu=1.0, n_samples=args.samples)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for i in range(args.warmup):
        tsx.is_fer_estimate(h, ts, stream=stream, job_key=10_000 + i, **kw)
    if dist:
        dist.barrier()
    ms, eu, nf, fer = [], 0, 0, []
    with Clocks(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            # the step's own job key: rank r, step i (independent sample streams)
            r = tsx.is_fer_estimate(h, ts, stream=stream, job_key=(rank << 32) | i, **kw)
            ms.append(r["ms"])
            eu += r["edge_updates"]
            nf += r["n_fail"]
            fer.append(r["fer"])
    clocks = clk.summary()
    total_ms = sum(ms)
    samples = float(args.samples) * args.steps
    if dist:
        total_ms, (samples, eu) = reduce_time_and_work(total_ms, [samples, eu], device="cuda")
    # end to end: the public call from host arrays (the set's nodes) to the host result
    t0 = time.perf_counter()
    tsx.is_fer_estimate(h, ts, stream=stream, job_key=99, **kw)
    e2e_s = time.perf_counter() - t0
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return None
    if pk is None:
        pk = tsx.measure_peaks()
    eu_launch = eu / args.steps if not dist else eu / world / args.steps
    line = {
        "metric": "importance-sampling samples/s",
        "value": samples / (total_ms / 1e3),
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int16",
        "data": "synthetic",
        "config": {"workload": "isfer", "code": code.name, "n": code.n, "m": code.m, "a": len(ts),
                   "ebn0_db": 4.0, "mu": 1.0, "samples_per_step": args.samples, "K": 20,
                   "parallelism": f"replicas{world}", "l2": "flushed before each step (256 MB write)"},
        "edge_updates_per_s": eu / (total_ms / 1e3),
        "fer_mean": float(np.mean(fer)), "fails_per_step": nf / args.steps,
        "roofline": alu_roofline(eu_launch, sum(ms) / len(ms), pk, clocks.get("sm_mhz"),
                                 note="edge updates of the decodes against the decoders' bound; the noise "
                                      "generation is extra work not counted"),
        "cpu_baseline": None,
        "e2e": {"value": args.samples / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": 4 * len(ts),
                "d2h_bytes_per_step": 96},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return line


def _timed(fn, stream):
    """Device milliseconds of fn() on `stream` (CUDA events), after a 256 MB L2 flush."""
    import torch
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        flush.fill_(1)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def extra_list(tsx, pk, stream, steps=2, limit=-1):
    """The ordered list of Sec. III on the 2640-node QC code (every canonical
    candidate, K = 100): first stage (the enumeration decode) and second stage
    (replay and sieve of every x_k from ceil(average converged iterations))."""
    w = synth.workload("qc2640")
    c = tsx.load_code(w["code"], stream=stream)
    p = params_of(w, "nms16")
    if limit >= 0:
        p["cand_end"] = limit
    for _ in range(1):
        tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, list_mode=1, kstart=-1, **p))
    rows = []
    for _ in range(steps):
        ms, st = _timed(lambda: tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, list_mode=1, kstart=-1, **p)),
                        stream)
        rows.append((ms, st))
    ms = statistics.median(r[0] for r in rows)
    st = rows[-1][1]
    single = tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, **p))
    return {"workload": "qc2640 list mode (two-stage, kstart = ceil(avg))", "ms_per_step": ms,
            "n_cand": st["n_cand"], "n_ts": st["n_ts"], "n_ts_single_pattern": single["n_ts"],
            "distinct_ts_per_s": st["n_ts"] / (ms / 1e3), "list_kstart": st["list_kstart"],
            "list_patterns": st["list_patterns"], "ms_first_stage": st["ms_decode"],
            "ms_second_stage": st["ms_sieve"], "second_stage_iterations": st["list_iterations"],
            "edge_updates_per_s": (st["edge_updates"] + st["list_iterations"] * w["code"].E) / (ms / 1e3),
            "gpu_launches": 3 + 3 + 1 + 1 + 2}


def extra_budget(tsx, pk, stream):
    """Cycle-density iteration budgets (Sec. III, Table V) on Code 1 of Table V
    (girth 4; the PEG code has girth 8, so no 4- or 6-cycles and no budget):
    every candidate of size 1-2, K = 50, s = 12, against
    K(I) = 10 + ceil(40 * 4 / (4 + W(I)))."""
    E, Z = _code1()
    c = tsx.load_code(synth.qc_code(E, Z), stream=stream)
    p = dict(decoder="nms16", K=50, base_llr=16, amp_steps=12, max_size=2, cycle_len=0)
    out = {}
    for name, extra in (("plain", {}), ("budget", dict(budget_wref=4, budget_kmin=10))):
        tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, **p, **extra))
        ms, st = _timed(lambda: tsx.ts_list_view(tsx.enumerate_ts(c, stream=stream, **p, **extra)), stream)
        out[name] = {"ms": ms, "edge_updates": st["stats"]["edge_updates"], "n_ts": st["stats"]["n_ts"],
                     "n_cand": st["stats"]["n_cand"], "keys": set(st["keys"])}
    kp, kb = out["plain"].pop("keys"), out["budget"].pop("keys")
    return {"workload": "Code 1 (Table V), candidates of size 1-2, K 50, s 12, with and without iteration budgets "
                        "(wref 4, kmin 10)", **out,
            "speedup": out["plain"]["ms"] / out["budget"]["ms"],
            "edge_update_ratio": out["budget"]["edge_updates"] / max(1, out["plain"]["edge_updates"]),
            "sets_kept": len(kp & kb) / max(1, len(kp)), "sets_new": len(kb - kp)}


# single-precision operations of one sum-product edge update, counted from
# the decoder's series (IEEE-rounded adds, multiplies and divides, no fused
# multiply-add): tanh of q/2 (range reduction, the degree-9 expm1 Horner
# sum, e / (e + 2): about 42), the product over the other d - 1 = 5 edges
# (5), atanh of the product (series or frexp/log series, about 30), the
# clips, x2 and the variable-node add and extrinsic subtract (about 7)
SPA_OPS_PER_EDGE = 84


def extra_spa(tsx, pk, stream, sm_mhz):
    """The single-precision sum-product decoder on the PEG code's first
    200,000 candidates (K = 50, 12 halvings of the amplitude)."""
    w = synth.workload("peg1008")
    c = tsx.load_code(w["code"], stream=stream)
    p = dict(params_of(w, "spa"), cand_end=200_000)
    tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, **p))
    ms, st = _timed(lambda: tsx.ts_list_stats(tsx.enumerate_ts(c, stream=stream, **p)), stream)
    mhz = sm_mhz or SM_MAX_MHZ
    peak = pk["fp32_fma_per_clk_sm"] * pk["num_sms"] * mhz * 1e6 / SPA_OPS_PER_EDGE
    achieved = st["edge_updates"] / (st["ms_decode"] / 1e3)
    return {"workload": "peg1008[:200000], single-precision sum-product, K 50, s 12", "ms_per_step": ms,
            "edge_updates_per_s": st["edge_updates"] / (ms / 1e3), "n_ts": st["n_ts"], "decodes": st["decodes"],
            "roofline": {"bound": "fp32", "achieved": achieved, "peak": peak, "unit": "edge-updates/s",
                         "frac": achieved / peak,
                         "note": f"{SPA_OPS_PER_EDGE} single-precision operations per edge update against the "
                                 "measured FP32 lane rate; decode kernel time"},
            "gpu_launches": 10}


def extra_lnms(tsx, pk, stream, sm_mhz):
    """The paper's simulation decoder (layered min-sum, 4/4/6 bits, 20
    iterations) on Code 1 of Table V ((2560, 2048), 4 x 20 base, Z = 128),
    200,000 frames at Eb/N0 = 3 dB."""
    E, Z = _code1()
    c = tsx.load_code(synth.qc_code(E, Z), stream=stream)
    kw = dict(ebn0_db=3.0, max_frames=200_000, max_errors=0)
    tsx.lnms_simulate(c, stream=stream, job_key=1, **kw)
    r = tsx.lnms_simulate(c, stream=stream, job_key=2, **kw)
    return {"workload": "Code 1 (Table V), 200,000 frames, 3 dB, LLR/C2V/V2C 4/4/6 bits, 20 iterations",
            "frames_per_s": r["frames"] / (r["ms"] / 1e3), "fer": r["fer"], "ber": r["ber"],
            "edge_updates_per_s": r["edge_updates"] / (r["ms"] / 1e3), "ms": r["ms"],
            "roofline": alu_roofline(r["edge_updates"], r["ms"], pk, sm_mhz, packed=False,
                                     note="one frame per group, 8-bit values, scalar integer operations"),
            "gpu_launches": -(-200_000 // 65536)}


def extra_emd(tsx, stream):
    """EMD spectrum of Code 1 (Table II) up to 12-cycles on the device."""
    E, Z = _code1()
    c = tsx.load_code(synth.qc_code(E, Z), stream=stream)
    tsx.emd_spectrum(c, 5, stream=stream)
    s = tsx.emd_spectrum(c, 6, stream=stream)
    rows = {f"{2 * l}": {str(e): float(s["count2l"][l, e]) / (2 * l) for e in np.flatnonzero(s["count2l"][l])}
            for l in range(2, 7)}
    return {"workload": "Code 1 (Table V), cycles of length 4..12", "ms": s["ms"],
            "walks": int(s["walks"].sum()), "spectrum_per_orbit": rows, "gpu_launches": 1}


def _code1():
    rows, Z = [], None
    with open(os.path.join(ROOT, "tests", "golden", "code1_table5.txt")) as f:
        for line in f:
            t = line.split("#", 1)[0].split()
            if not t:
                continue
            if t[0] == "Z":
                Z = int(t[1])
            elif t[0][0] in "-0123456789":
                rows.append([int(x) for x in t])
    return np.array(rows, dtype=np.int32), Z


def run_extras(args, tsx, pk):
    """The library's other workloads, a few steps each, summarized for the
    headline line (one GPU)."""
    import copy
    out = {}

    def sub(**kw):
        a = copy.copy(args)
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    keep = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config", "roofline", "e2e",
            "gpu_launches", "clocks")
    for name, fn, kw, more in (
            ("batch32", run_batch, dict(steps=3, warmup=3, tune=True, e2e_steps=1),
             ("serial_ms_per_step", "batch_speedup_vs_serial", "decodes_per_s", "n_ts")),
            ("serve", run_serve, dict(jobs=120, load=0.8),
             ("p50_ms", "p90_ms", "p99_ms", "mean_ms", "plain", "edge_updates_per_s", "makespan_ms",
              "max_concurrent_jobs", "hbm_peak_bytes", "results_identical_to_plain")),
            ("isfer", run_isfer, dict(steps=3, warmup=3, samples=1_000_000),
             ("edge_updates_per_s", "fer_mean", "fails_per_step"))):
        t0 = time.perf_counter()
        try:
            line = fn(sub(workload=name, **kw), pk) if fn is not run_serve else fn(sub(workload=name, **kw))
            out[name] = {k: line[k] for k in keep + more if k in line}
        except Exception as e:  # one workload's failure must not hide the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    import torch
    stream = torch.cuda.Stream()
    sm = None
    for name, fn in (("list_mode", lambda: extra_list(tsx, pk, stream)),
                     ("iteration_budget", lambda: extra_budget(tsx, pk, stream)),
                     ("layered_simulation", lambda: extra_lnms(tsx, pk, stream, sm)),
                     ("sum_product", lambda: extra_spa(tsx, pk, stream, sm)),
                     ("emd_spectrum", lambda: extra_emd(tsx, stream))):
        t0 = time.perf_counter()
        try:
            with Clocks(torch.cuda.current_device()) as clk:
                out[name] = fn()
            out[name]["clocks"] = clk.summary()
        except Exception as e:
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def run_extra_alone(args):
    import torch
    import paper_2208_05795_gb300 as tsx
    from paper_2208_05795_gb300 import build as tsx_build
    torch.cuda.set_device(0)
    tsx_build.build()
    pk = tsx.measure_peaks()
    stream = torch.cuda.Stream()
    fn = {"list2640": lambda: extra_list(tsx, pk, stream, steps=args.steps, limit=args.cand_limit),
          "budget_code1": lambda: extra_budget(tsx, pk, stream),
          "lnms_code1": lambda: extra_lnms(tsx, pk, stream, None),
          "emd_code1": lambda: extra_emd(tsx, stream),
          "spa_peg": lambda: extra_spa(tsx, pk, stream, None)}[args.workload]
    with Clocks(0) as clk:
        d = fn()
    metric, unit, key = EXTRA_WORKLOADS[args.workload]
    line = {"metric": metric, "value": d[key], "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": unit != "ms", "scaling": "weak", "vs_baseline": None,
            "data": "synthetic", "config": {"workload": args.workload}, **d, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    line = None
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in EXTRA_WORKLOADS:
        run_extra_alone(args)
        return
    if args.workload == "isfer":
        line = run_isfer(args)
    elif args.workload == "serve":
        line = run_serve(args)
    elif args.workload == "batch32":
        line = run_batch(args)
    else:
        run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
