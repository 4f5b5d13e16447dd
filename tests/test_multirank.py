"""Several ranks on CPU (gloo, world size 2): one code's candidate list split
into ranges, each range enumerated on its own rank, the trapping-set lists
merged by the exchange step, and the max-time / summed-work reduction that
bench.py uses.  The merged list must equal the whole-code enumeration.
The ranges are enumerated by the oracle here (no GPU); on GPUs the library
produces the same per-range records (tests/test_gpu_parity.py shards)."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import synth
from paper_2208_05795_gb300.shard import merge_records, shard_bounds

P = dict(K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)


def _oracle_records(res):
    return {t.key: (t.a, t.b, t.orbit, int(t.elementary), t.count, t.thr, float(t.thr_f)) for t in res.ts_list}


def test_shard_bounds_cover_exactly():
    for n in (0, 1, 7, 100, 9118):
        for world in (1, 2, 3, 8):
            ranges = [shard_bounds(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_bounds(10, 2, 2)


def test_merge_is_order_independent_and_checks_agreement():
    a = {(1, 2): (2, 2, 16, 1 | 2, 3, 40, -1.0), (5,): (1, 3, 16, 1 | 2, 1, 90, -1.0)}
    b = {(1, 2): (2, 2, 16, 1 | 4, 2, 35, -1.0), (7, 9): (2, 4, 8, 0 | 4, 1, -1, -1.0)}
    m1, m2 = merge_records([a, b]), merge_records([b, a])
    assert m1 == m2
    assert m1[(1, 2)] == (2, 2, 16, 7, 5, 35, -1.0)
    bad = {(1, 2): (3, 2, 16, 1, 1, 10, -1.0)}
    with pytest.raises(ValueError):
        merge_records([a, bad])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    from paper_2208_05795_gb300.shard import exchange, reduce_time_and_work
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = oracle.Graph(synth.workload("qc96")["code"])
        cands = g.candidates(P["max_size"], P["cycle_len"])
        b, e = shard_bounds(len(cands), rank, world)
        res = g.enumerate(cands[b:e], **P)
        merged = exchange(_oracle_records(res))
        ms, work = reduce_time_and_work(10.0 * (rank + 1), [rank + 1, len(res.ts_list)])
        if rank == 0:
            with open(out_path, "wb") as f:
                pickle.dump((merged, ms, work), f)
    finally:
        dist.destroy_process_group()


def test_two_ranks_merge_equals_whole_code(tmp_path):
    out = str(tmp_path / "rank0.pkl")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    with open(out, "rb") as f:
        merged, ms, work = pickle.load(f)
    g = oracle.Graph(synth.workload("qc96")["code"])
    whole = _oracle_records(g.enumerate(**P))
    assert merged == whole
    assert ms == 20.0
    assert work[0] == 3.0 and work[1] >= len(whole)
    assert np.isfinite(ms)
