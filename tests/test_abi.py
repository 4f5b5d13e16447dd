"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/*.h declares (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

import helpers  # noqa: F401  (sys.path set by conftest)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = "\n".join(l for l in text.splitlines() if not l.lstrip().startswith("#"))
        for m in re.finditer(r"TSX_API\s+[^;]*?\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.S):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2208_05795_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for fn in ("load_code", "free_code", "enumerate_ts", "free_ts_list", "ts_list_view", "tsx_strerror"):
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_without_gpu(libpath):
    import paper_2208_05795_gb300 as tsx
    assert tsx.strerror(-2).startswith("out of memory")
    p = tsx.enum_params_default()
    assert (p.K, p.base_llr, p.sat, p.alpha_num, p.alpha_shift, p.amp_steps) == (20, 16, 511, 3, 2, 10)
    q = tsx.make_params(decoder="spa", K=50, amp_steps=12)
    assert (q.decoder, q.K, q.amp_steps) == (2, 50, 12)
    with pytest.raises(TypeError):
        tsx.make_params(bogus=1)


def test_view_marshalling_keys_as_arrays_and_tuples():
    # the binding's copy of a ts_list_view() result (no library call): the
    # canonical keys come back as one concatenated array with offsets, and
    # with keys=True also as tuples equal to the slices
    import numpy as np
    from paper_2208_05795_gb300 import _tsx

    def ptr(a, t):
        return a.ctypes.data_as(ctypes.POINTER(t))

    off = np.array([0, 3, 3, 7], np.int64)  # a set of size 0 is kept as an empty key
    vars_ = np.array([5, 9, 11, 0, 2, 4, 1000], np.int32)
    per_ts = {k: np.arange(3, dtype=np.int32) + i for i, k in enumerate(("a", "b", "orbit", "count", "thr", "flags"))}
    thr_f = np.array([0.5, -1.0, 2.0], np.float32)
    cand = np.arange(8, dtype=np.int32)
    v = _tsx.TsView()
    v.n_ts, v.n_cand = 3, 2
    for k, arr in per_ts.items():
        setattr(v, k, ptr(arr, ctypes.c_int32))
    v.thr_f, v.var_off, v.vars = ptr(thr_f, ctypes.c_float), ptr(off, ctypes.c_int64), ptr(vars_, ctypes.c_int32)
    v.cand_vars = ptr(cand, ctypes.c_int32)
    for k in ("cand_thr", "cand_ts", "cand_flags", "cand_decodes", "cand_iters"):
        setattr(v, k, ptr(cand, ctypes.c_int32))
    v.cand_thr_f = ptr(thr_f, ctypes.c_float)
    with_keys = _tsx._view_dict(v, 0, True)
    without = _tsx._view_dict(v, 0, False)
    assert with_keys["keys"] == [(5, 9, 11), (), (0, 2, 4, 1000)]
    assert "keys" not in without
    for d in (with_keys, without):
        assert np.array_equal(d["key_vars"], vars_) and np.array_equal(d["key_off"], off)
        assert np.array_equal(d["orbit"], per_ts["orbit"]) and d["cand_vars"].shape == (2, 4)
