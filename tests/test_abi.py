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
