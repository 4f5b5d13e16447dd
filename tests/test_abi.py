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
