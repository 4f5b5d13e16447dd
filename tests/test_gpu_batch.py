"""GPU: batches of codes in one multi-code decode launch, replayed from a
CUDA graph, and the tile autotuner.

A batch must give, code by code, exactly what enumerate_ts gives for that
code alone (which the parity tests pin to the oracle), whatever the other
codes in the batch, the tile, the message storage or the way it is launched
(eagerly, re-run, or replayed from a captured graph).  One code of the batch
is also compared with the oracle directly.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2208_05795_gb300 as tsx
from gpu_helpers import lib_records, lib_ts, oracle_records, oracle_ts
from test_gpu_parity import _sampled_compare, _ts_invariants

pytestmark = pytest.mark.gpu

P2 = dict(K=20, base_llr=16, amp_steps=10, max_size=2, cycle_len=0)
ARRAYS = ("a", "b", "orbit", "count", "thr", "thr_f", "flags", "cand_vars", "cand_thr", "cand_thr_f", "cand_ts",
          "cand_flags", "cand_decodes", "cand_iters")


def _same(v, w):
    assert v["keys"] == w["keys"]
    for k in ARRAYS:
        assert np.array_equal(v[k], w[k]), k
    for k in ("n_cand", "n_cand_total", "n_ts", "decodes", "iterations", "edge_updates", "acyclic"):
        assert v["stats"][k] == w["stats"][k], k


def _single(code, params):
    lst = tsx.enumerate_ts(code, params)
    return tsx.ts_list_view(lst)


@pytest.fixture(scope="module")
def small_batch():
    # the tiny 3x6 code and three 4 x n_b codes of uneven sizes (check degrees 6 .. 28)
    codes = [synth.workload("qc96")["code"]] + synth.batch_codes([102, 112, 116])
    return [tsx.load_code(c) for c in codes], codes


def test_batch_equals_single(small_batch):
    handles, _ = small_batch
    b = tsx.batch_create(handles, P2)
    assert len(b) == len(handles) and b.multi_launch
    tsx.batch_run(b)
    for i, h in enumerate(handles):
        _same(tsx.batch_view(b, i), _single(h, tsx.make_params(**P2)))


def test_batch_rerun_and_mixed_params(small_batch):
    handles, codes = small_batch
    # per-code parameters: the tiny code with the full size-3 candidate rule
    ps = [tsx.make_params(**dict(P2, max_size=3))] + [tsx.make_params(**dict(P2, K=15))] * (len(handles) - 1)
    b = tsx.batch_create(handles, ps)
    tsx.batch_run(b)
    first = [tsx.batch_view(b, i) for i in range(len(handles))]
    tsx.batch_run(b)
    for i in range(len(handles)):
        _same(tsx.batch_view(b, i), first[i])
    # the tiny code against the oracle in full
    g = oracle.Graph(codes[0])
    res = g.enumerate(K=20, base_llr=16, amp_steps=10, max_size=3, cycle_len=0)
    assert len(first[0]["cand_thr"]) == 9118
    assert lib_records(first[0]) == oracle_records(res)
    assert lib_ts(first[0]) == oracle_ts(res)
    for i in range(1, len(handles)):
        _same(first[i], _single(handles[i], ps[i]))


def test_batch_sampled_oracle(small_batch):
    handles, codes = small_batch
    b = tsx.batch_create(handles, P2)
    tsx.batch_run(b)
    v = tsx.batch_view(b, 2)
    w = dict(code=codes[2], **P2)
    g = _sampled_compare(w, v, 40, seed=5)
    _ts_invariants(g, v, qc=True)


def test_batch_graph_replay(small_batch):
    handles, _ = small_batch
    side = torch.cuda.Stream()
    b = tsx.batch_create(handles, P2, stream=side)
    with torch.cuda.stream(side):
        tsx.batch_run(b, stream=side)
    side.synchronize()
    eager = [tsx.batch_view(b, i) for i in range(len(handles))]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        tsx.batch_run(b, stream=torch.cuda.current_stream())
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for i in range(len(handles)):
            _same(tsx.batch_view(b, i), eager[i])


def test_batch_fallback_per_code_launches(small_batch):
    handles, _ = small_batch
    b = tsx.batch_create(handles, tsx.make_params(**dict(P2, kernel=1)))
    assert not b.multi_launch
    tsx.batch_run(b)
    for i, h in enumerate(handles):
        _same(tsx.batch_view(b, i), _single(h, tsx.make_params(**P2)))


@pytest.mark.parametrize("sat", [511, 150])
def test_tune_tile_keeps_results(small_batch, sat):
    handles, _ = small_batch
    base = tsx.make_params(**dict(P2, sat=sat))
    tuned = []
    for h in handles:
        t, ms = tsx.tune_tile(h, base)
        assert ms > 0.0
        assert t.warps_per_cta in (0, 1, 2, 4, 8)  # 0: the automatic shape
        assert t.decoder in (0, 1) and (sat <= 169 or t.decoder == 0)
        tuned.append(t)
    if sat <= 169:
        # force int8 storage on one code: the results may not change
        tuned[1].decoder = tsx.DECODERS["nms8"]
    ref = [_single(h, base) for h in handles]
    for i, h in enumerate(handles):
        _same(_single(h, tuned[i]), ref[i])
    # a batch needs one message storage for all codes
    for t in tuned:
        t.decoder = tuned[1].decoder
    b = tsx.batch_create(handles, tuned)
    assert b.multi_launch
    tsx.batch_run(b)
    for i in range(len(handles)):
        _same(tsx.batch_view(b, i), ref[i])


def test_batch_with_code_too_large_for_the_pair_layout():
    # n = 11520 (4 x 30 base, Z = 384): its two-codeword layout does not fit
    # one CTA's shared memory, so it is decoded by a launch of its own
    codes = [synth.workload("qc96")["code"]] + synth.batch_codes([122, 116])
    handles = [tsx.load_code(c) for c in codes]
    ps = [tsx.make_params(**P2), tsx.make_params(**dict(P2, cand_end=3000)), tsx.make_params(**P2)]
    b = tsx.batch_create(handles, ps)
    assert b.multi_launch
    tsx.batch_run(b)
    for i, h in enumerate(handles):
        _same(tsx.batch_view(b, i), _single(h, ps[i]))
