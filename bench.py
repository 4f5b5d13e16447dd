#!/usr/bin/env python
"""Benchmark: impulse-decode edge-updates/s of the trapping-set enumeration.

One step = one enumerate_ts() call on the workload: candidate generation and
canonical dedupe, impulse decodes with amplitude bisection, sieving,
classification, canonical form and dedupe of the trapping sets -- the whole
hot path -- over every canonical candidate of the code.  Inputs (the code's
device tables) are resident when the timed region starts; L2 is flushed
(a 256 MB write) before every timed step, outside its CUDA-event bracket.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank enumerates its own code of the same shape
(rank r uses seed offset r: independent problems, weak scaling); no
collective on the data path, a barrier and max-over-ranks time only.
--impl reference times the CPU oracle (single thread) on a bounded sample
of the same workload each step.
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

# integer operations the min-sum edge update needs at minimum: |q|, two
# compare-selects for min1/min2, argmin select, sign xor, output select,
# x3, >>2, sign apply, the add of the variable-node sum, the subtract of
# P - r and the two-sided clamp (counted as one)
ALG_OPS_PER_EDGE = 12
# INT32 lanes per SM that execute IADD3/LOP3 each clock (Blackwell SM: 4
# partitions x 32 lanes); with 152 SMs at the 2070 MHz maximum SM clock.
INT_LANES_PER_SM = 128
N_SMS = 152
SM_MAX_MHZ = 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="peg1008", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--decoder", default="nms16", choices=["nms16", "nms8", "spa"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--cand-limit", type=int, default=-1,
                    help="decode only the first N canonical candidates (profiling a bounded case)")
    return ap.parse_args()


def rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def workload_for(name, rank):
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


def cpu_baseline(w, decoder, seconds, rng_seed=0):
    """The oracle (single thread, as it stands) on a bounded random sample of
    the workload's canonical candidates; edge-updates/s."""
    import oracle
    g = oracle.Graph(w["code"])
    cands = g.candidates(w["max_size"], w["cycle_len"])
    rng = np.random.default_rng(rng_seed)
    p = params_of(w, decoder)
    p.pop("decoder")
    od = "spa" if decoder == "spa" else "nms"
    extra = dict(sat=127) if decoder == "nms8" else {}
    n, it, el, ncand = 4, 0, 0.0, 0
    while el < seconds:
        pick = rng.choice(len(cands), min(n, len(cands)), replace=False)
        t0 = time.perf_counter()
        res = g.enumerate(cands[np.sort(pick)], decoder=od, **p, **extra)
        el += time.perf_counter() - t0
        it += int(res.iters.sum())
        ncand += len(pick)
        n = min(len(cands), n * 2)
    return {"value": it * g.E / el, "unit": "edge-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{ncand} random canonical candidates of {len(cands)} (seeded), "
                      f"{el:.1f} s single-threaded"}, ncand / el


def run_reference(args):
    rank, world, _ = rank_world()
    if rank != 0:
        return
    w = workload_for(args.workload, 0)
    base, _ = cpu_baseline(w, args.decoder, max(2.0, args.cpu_seconds / 3))
    times, eus = [], []
    import oracle
    g = oracle.Graph(w["code"])
    cands = g.candidates(w["max_size"], w["cycle_len"])
    p = params_of(w, args.decoder)
    p.pop("decoder")
    od = "spa" if args.decoder == "spa" else "nms"
    rng = np.random.default_rng(1)
    per_step = max(8, int(len(cands) / 2000))
    per_step = min(per_step, 64)
    for s in range(args.warmup + args.steps):
        pick = np.sort(rng.choice(len(cands), per_step, replace=False))
        t0 = time.perf_counter()
        res = g.enumerate(cands[pick], decoder=od, **p)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            eus.append(int(res.iters.sum()) * g.E)
    value = sum(eus) / sum(times)
    line = {"impl": "reference", "metric": "impulse-decode edge-updates/s", "value": value,
            "unit": "edge-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.decoder == "spa" else "int16", "data": "synthetic",
            "config": {"workload": args.workload, "decoder": args.decoder,
                       "sample_per_step": per_step, "n_cand": int(len(cands))},
            "cpu_baseline": {"value": value, "unit": "edge-updates/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} random canonical candidates per step"},
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
    w = workload_for(args.workload, rank)
    params = params_of(w, args.decoder)
    if args.decoder == "nms8":
        params["sat"] = 127
    if args.cand_limit >= 0:
        params["cand_end"] = args.cand_limit
    stream = torch.cuda.Stream()
    code = tsx.load_code(w["code"], stream=stream)
    info = code.info
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    has_cycles = w["cycle_len"] // 2 > w["max_size"]
    launches_per_step = 3 + (3 if has_cycles else 0) + 1 + 2

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
        t = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        e = torch.tensor([eu, dec], dtype=torch.float64, device="cuda")
        dist.all_reduce(e)
        eu_all, dec_all = float(e[0].item()), float(e[1].item())
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
            v = tsx.ts_list_view(tsx.enumerate_ts(c2, stream=stream, **params))
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            eu2 += v["stats"]["edge_updates"]
            n_rep = c2.info["n_rep"]
            h2d = desc_bytes + 8 * (n_rep + 1)
            d2h = sum(v[k].nbytes for k in ("cand_vars", "cand_thr", "cand_thr_f", "cand_ts", "cand_flags",
                                            "cand_decodes", "cand_iters", "a", "b", "orbit", "count", "thr",
                                            "flags", "thr_f")) + 4 * sum(len(k) + 4 for k in v["keys"])
            del c2
        e2e = {"value": eu2 / wall, "unit": "edge-updates/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak = INT_LANES_PER_SM * N_SMS * SM_MAX_MHZ * 1e6 / 1e12  # Tops/s
    avg_dec_ms = sum(ms_dec) / len(ms_dec)
    eu_per_step = eu / args.steps
    achieved = ALG_OPS_PER_EDGE * eu_per_step / (avg_dec_ms / 1e3) / 1e12
    cpu = cpu_baseline(w, args.decoder, args.cpu_seconds)[0] if args.cpu_seconds > 0 else None
    line = {
        "metric": "impulse-decode edge-updates/s",
        "value": value,
        "unit": "edge-updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.decoder == "spa" else ("int8" if args.decoder == "nms8" else "int16"),
        "data": "synthetic",
        "config": {"workload": args.workload + (f"[:{args.cand_limit}]" if args.cand_limit >= 0 else ""),
                   "decoder": args.decoder, "n": info["n"], "m": info["m"],
                   "E": info["E"], "girth": info["girth"], "K": w["K"], "amp_steps": w["amp_steps"],
                   "base_llr": w["base_llr"], "n_cand": int(s["n_cand"]), "parallelism": f"replicas{world}",
                   "l2": "flushed before each step (256 MB write)"},
        "decodes_per_s": dec_all / (total_ms / 1e3),
        "distinct_ts_per_s": nts * world / (total_ms / args.steps / 1e3),
        "n_ts": nts,
        "ms_decode_kernel": avg_dec_ms,
        "ms_candidates": sum(ms_cand) / len(ms_cand),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": f"{ALG_OPS_PER_EDGE} int ops per edge update; peak = {INT_LANES_PER_SM} lanes x "
                             f"{N_SMS} SMs x {SM_MAX_MHZ:.0f} MHz"},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
