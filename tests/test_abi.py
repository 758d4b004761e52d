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


def test_struct_layout_matches_header(tmp_path):
    """The binding's ctypes mirrors of the header's structs have the C
    compiler's sizes and field offsets (a field added to one side only would
    shift every later field and every result of a batch)."""
    import subprocess
    import paper_1304_5966_gb300 as sw
    structs = {"sw_scheme": sw._Scheme, "sw_stats": sw._Stats, "sw_result": sw._Result, "sw_pair": sw._Pair}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "swgb.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in structs.items():
        assert int(got[f"{cname} size"]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname} {f}"]) == getattr(py, f).offset, (cname, f)


def test_batch_results_view_reads_every_field():
    """The bulk numpy view over a result array reads score, coordinates, cell
    count and strand at the C offsets (no GPU: results without CIGARs)."""
    import paper_1304_5966_gb300 as sw
    outs = (sw._Result * 3)()
    for k in range(3):
        outs[k].score, outs[k].a_begin, outs[k].a_end = 10 * k + 1, k, k + 5
        outs[k].b_begin, outs[k].b_end, outs[k].strand = 2 * k, 2 * k + 7, k % 2
        outs[k].stats.cells = 1000 + k
    outs[0].stats.tuned, outs[0].stats.band_rows = 1, 1024
    res = sw._batch_results(outs, 3)
    assert [(r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.strand) for r in res] == \
        [(1, 0, 5, 0, 7, 0), (11, 1, 6, 2, 9, 1), (21, 2, 7, 4, 11, 0)]
    assert res[0].stats["tuned"] == 1 and res[0].stats["band_rows"] == 1024 and res[0].cigar is None
    assert res[1].stats == {"cells": 1001} and res[2].stats == {"cells": 1002}
