"""C-ABI library checks that need no GPU: it builds, loads and exports every
function that include/swgb.h declares; error strings are defined."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1304_5966_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"sw_score", "sw_align", "sw_align_batch", "sw_ctx_create"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_strerror(lib):
    lib.sw_strerror.restype = ctypes.c_char_p
    assert lib.sw_strerror(0) == b"ok"
    assert lib.sw_strerror(4) == b"device-side wait timed out"


def test_null_arguments_are_rejected(lib):
    # no context: every entry point refuses before touching the GPU
    assert lib.sw_score(None, None, 0, None, 0, None, 0, None) == 1
    assert lib.sw_align(None, None, 0, None, 0, None, 0, None) == 1
    assert lib.sw_align_batch(None, None, 0, None, 0, None) == 1
    assert lib.sw_ctx_set_option(None, 1, 16) == 1
