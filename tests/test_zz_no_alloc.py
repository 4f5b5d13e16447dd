"""decode_thresholds_noalloc(): the impulse decoder for callers that cannot
allocate device memory (it keeps its working memory in one fixed device
array inside the library).  Its per-candidate results must equal those of
enumerate_ts() on the same candidate sets -- bit for bit, as every decoder
test here requires -- on two calls in a row, the second of which finds the
first call's leftovers in the shared array.  The test itself allocates its
input and output buffers with torch; the entry point under test does not."""
import numpy as np
import pytest

import paper_2208_05795_gb300 as tsx
import synth

pytestmark = pytest.mark.gpu

TSX_ENOMEM, TSX_EINVAL = -2, -1


def _params(w, **over):
    p = dict(K=w["K"], base_llr=w["base_llr"], amp_steps=w["amp_steps"], max_size=w["max_size"],
             cycle_len=w["cycle_len"])
    p.update(over)
    return p


def _noalloc(code, cand, params, check=True):
    import torch
    n = cand.shape[0]
    c = torch.from_numpy(np.ascontiguousarray(cand, dtype=np.int32)).cuda()
    thr = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    thr_f = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
    dec = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    it = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = tsx.decode_thresholds_noalloc(code, c.data_ptr(), n, thr.data_ptr(), thr_f.data_ptr(), dec.data_ptr(),
                                       it.data_ptr(), check=check, **params)
    torch.cuda.synchronize()
    return st, thr.cpu().numpy(), thr_f.cpu().numpy(), dec.cpu().numpy(), it.cpu().numpy()


@pytest.mark.parametrize("decoder", ["nms16", "spa"])
def test_noalloc_equals_enumerate_ts_on_two_calls(decoder):
    import torch
    assert torch.cuda.is_available()
    w = synth.workload("qc96")
    p = _params(w, decoder=decoder, amp_steps=12 if decoder == "spa" else w["amp_steps"])
    code = tsx.load_code(w["code"])
    v = tsx.ts_list_view(tsx.enumerate_ts(code, **p))
    cand = v["cand_vars"]
    # call 1: every candidate; call 2: a reversed subset (the array still
    # holds call 1's counters and patterns)
    _, thr, thr_f, dec, it = _noalloc(code, cand, p)
    assert np.array_equal(thr, v["cand_thr"])
    assert np.array_equal(thr_f, v["cand_thr_f"])
    assert np.array_equal(dec, v["cand_decodes"])
    assert np.array_equal(it, v["cand_iters"])
    sel = np.arange(len(cand))[::-3]
    _, thr2, thr_f2, dec2, it2 = _noalloc(code, cand[sel], p)
    assert np.array_equal(thr2, v["cand_thr"][sel])
    assert np.array_equal(thr_f2, v["cand_thr_f"][sel])
    assert np.array_equal(dec2, v["cand_decodes"][sel])
    assert np.array_equal(it2, v["cand_iters"][sel])


def test_noalloc_limits_and_bad_input():
    w = synth.workload("qc96")
    p = _params(w)
    code = tsx.load_code(w["code"])
    cand = np.array([[0, 1, -1, -1]], dtype=np.int32)
    # beyond the fixed scratch: refused before any work
    import torch
    c = torch.from_numpy(cand).cuda()
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = tsx.decode_thresholds_noalloc(code, c.data_ptr(), 10 ** 9, out.data_ptr(), None, out.data_ptr(),
                                       out.data_ptr(), check=False, **p)
    assert st == TSX_ENOMEM
    # a count whose byte size would wrap a 64-bit size: refused the same way
    st = tsx.decode_thresholds_noalloc(code, c.data_ptr(), 2 ** 62, out.data_ptr(), None, out.data_ptr(),
                                       out.data_ptr(), check=False, **p)
    assert st == TSX_ENOMEM
    # a node index outside the code is caught by the device-side check
    st, *_ = _noalloc(code, np.array([[0, 96, -1, -1]], dtype=np.int32), p, check=False)
    assert st == TSX_EINVAL
    st, *_ = _noalloc(code, np.array([[-1, 3, -1, -1]], dtype=np.int32), p, check=False)
    assert st == TSX_EINVAL
    # and the entry point still works afterwards
    st, thr, *_ = _noalloc(code, cand, p)
    assert st == 0 and thr[0] >= -1
