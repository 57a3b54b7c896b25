"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no GPU needed: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1512_01641_gb300 import build, miner

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["mine_plan_create", "mine_pairs", "mine_count", "mine_align", "mine_score", "mine_strerror"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for n in _declared():
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_binding_signatures_cover_header(libpath):
    assert set(_declared()) <= set(miner._SIGS), set(_declared()) - set(miner._SIGS)


def test_strerror_without_gpu(libpath):
    L = miner.lib()
    assert L.mine_strerror(0) == b"ok"
    assert b"invalid" in L.mine_strerror(-1)
    assert L.mine_strerror(-4).startswith(b"device-side wait")


@pytest.mark.parametrize("opts", [
    [(99, 1)],                       # unknown option
    [(7, 0)],                        # MINE_OPT_GRAPH_CAPTURES is read-only
    [(9, 0)],                        # MINE_OPT_N_TILE_FLAGS is read-only
    [(1, 48)],                       # tile width not a multiple of 32
    [(1, 64), (2, 0)],               # a valid option followed by an invalid one
    [(10, 4)],                       # soft split mode out of range
])
def test_create_with_options_rejects_bad_options_before_device_work(libpath, opts):
    # option validation comes before any CUDA call, so this runs without a GPU;
    # the corpora only need non-null pointers to reach it
    L = miner.lib()
    buf = (ctypes.c_int64 * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    src = miner._Corpus(1, 1, 1, p, p, p)
    tgt = miner._Corpus(1, 1, 1, p, p, p)
    dic = miner._Dict(4, 4, 1, p, p)
    ids = (ctypes.c_int32 * len(opts))(*[o for o, _ in opts])
    vals = (ctypes.c_int64 * len(opts))(*[v for _, v in opts])
    h = ctypes.c_void_p()
    rc = L.mine_plan_create_with_options(ctypes.byref(src), ctypes.byref(tgt), ctypes.byref(dic), ids, vals,
                                         len(opts), ctypes.byref(h), None)
    assert rc == miner.MINE_EINVAL and not h.value
    rc = L.mine_plan_create_with_options(ctypes.byref(src), ctypes.byref(tgt), ctypes.byref(dic), ids, vals, -1,
                                         ctypes.byref(h), None)
    assert rc == miner.MINE_EINVAL and not h.value
