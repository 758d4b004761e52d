"""CPU oracle for exact affine-gap Smith-Waterman (test infrastructure only).

Only the test-suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  The library's product path never touches it; the
two share no code (the seeded input generator in ``gen/`` serves both and holds
none of the method's arithmetic).

The arithmetic lives in ``sw_oracle.c`` (plain scalar C, 64-bit integers);
this module compiles it with gcc on first use (or from ``build()``) and wraps
it with ctypes.  ``brute.py`` holds an exhaustive enumerator for tiny pairs
that pins the C code.

Paper: Korpar & Sikic, "SW# - GPU enabled exact alignments on genome scale",
Sec. 2 (Methods): score and end point by Smith-Waterman with affine gaps, start
point by the modified reverse pass, alignment between them by Needleman-Wunsch.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsworacle.so")

H, E, F = 0, 1, 2          # node states (E horizontal / 'D', F vertical / 'I')


@dataclass(frozen=True)
class Scheme:
    """Substitution scores and affine gap costs; gap of length k = go + ge*(k-1)."""
    match: int = 1
    mismatch: int = -3
    gap_open: int = 5
    gap_extend: int = 2
    alphabet: int = 4
    matrix: tuple | None = None     # alphabet*alphabet row-major, overrides match/mismatch

    def table(self) -> np.ndarray:
        if self.matrix is not None:
            t = np.asarray(self.matrix, dtype=np.int32).reshape(self.alphabet, self.alphabet)
            return np.ascontiguousarray(t)
        t = np.full((self.alphabet, self.alphabet), self.mismatch, dtype=np.int32)
        for c in range(min(self.alphabet, 4)):
            t[c, c] = self.match          # code 4 (N) mismatches everything, itself included
        return t

    def max_sub(self) -> int:
        return int(self.table().max())


DNA = Scheme()


def build(force: bool = False) -> str:
    """Compile sw_oracle.c into _build/libsworacle.so (plain gcc -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, P = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        pi64 = ctypes.POINTER(ctypes.c_int64)
        lib.orc_local_score.restype = i64
        lib.orc_local_score.argtypes = [P, i64, P, i64, P, i32, i32, i32, pi64, pi64]
        lib.orc_reverse_start.restype = ctypes.c_int
        lib.orc_reverse_start.argtypes = [P, P, i64, i64, P, i32, i32, i32, i64, i32, pi64, pi64, pi64]
        lib.orc_global_trace.restype = i64
        lib.orc_global_trace.argtypes = [P, i64, P, i64, P, i32, i32, i32, i32, i32, P, i64, pi64]
        lib.orc_rescore.restype = i64
        lib.orc_rescore.argtypes = [P, P, P, i64, P, i32, i32, i32, i32, pi64, pi64]
        lib.orc_verify_path.restype = ctypes.c_int
        lib.orc_verify_path.argtypes = [P, i64, P, i64, P, i32, i32, i32, i32, i32, P, i64]
        lib.orc_local_matrix.restype = ctypes.c_int
        lib.orc_local_matrix.argtypes = [P, i64, P, i64, P, i32, i32, i32, P]
        _lib = lib
    return _lib


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _ptr(arr: np.ndarray):
    return arr.ctypes.data_as(ctypes.c_void_p)


def local_score(a, b, sch: Scheme = DNA):
    """(S, a_end, b_end): best local score and its end point (first in row-major order)."""
    a, b, t = _u8(a), _u8(b), sch.table()
    ei, ej = ctypes.c_int64(), ctypes.c_int64()
    s = _L().orc_local_score(_ptr(a), len(a), _ptr(b), len(b), _ptr(t), sch.alphabet,
                             sch.gap_open, sch.gap_extend, ctypes.byref(ei), ctypes.byref(ej))
    if s < 0:
        raise MemoryError("oracle allocation failed")
    return int(s), int(ei.value), int(ej.value)


def reverse_start(a, b, a_end: int, b_end: int, S: int, sch: Scheme = DNA, scan_all: bool = False):
    """(a_begin, b_begin, max_value) from the reverse anchored pass."""
    a, b, t = _u8(a), _u8(b), sch.table()
    bi, bj, mx = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = _L().orc_reverse_start(_ptr(a), _ptr(b), a_end, b_end, _ptr(t), sch.alphabet,
                                sch.gap_open, sch.gap_extend, S, int(scan_all),
                                ctypes.byref(bi), ctypes.byref(bj), ctypes.byref(mx))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    if rc != 0:
        raise RuntimeError("reverse pass found no cell with value S")
    return int(bi.value), int(bj.value), int(mx.value)


def global_trace(a, b, sch: Scheme = DNA, src: int = H, snk: int = H):
    """(value, ops) of the greedy-traceback global alignment from node src to node snk."""
    a, b, t = _u8(a), _u8(b), sch.table()
    cap = len(a) + len(b) + 8
    buf = ctypes.create_string_buffer(cap)
    v = ctypes.c_int64()
    n = _L().orc_global_trace(_ptr(a), len(a), _ptr(b), len(b), _ptr(t), sch.alphabet,
                              sch.gap_open, sch.gap_extend, src, snk, buf, cap, ctypes.byref(v))
    if n == -3:
        raise ValueError("sink unreachable from source")
    if n < 0:
        raise MemoryError(f"oracle global_trace failed ({n})")
    return int(v.value), buf.raw[:n].decode()


def rescore(a, b, ops: str, sch: Scheme = DNA, src: int = H):
    """(score, used_a, used_b) of an explicit op string over a, b."""
    a, b, t = _u8(a), _u8(b), sch.table()
    o = ops.encode()
    ua, ub = ctypes.c_int64(), ctypes.c_int64()
    s = _L().orc_rescore(_ptr(a), _ptr(b), o, len(o), _ptr(t), sch.alphabet,
                         sch.gap_open, sch.gap_extend, src, ctypes.byref(ua), ctypes.byref(ub))
    return int(s), int(ua.value), int(ub.value)


def verify_path(a, b, ops: str, sch: Scheme = DNA, src: int = H, snk: int = H) -> int:
    """0 if ops is exactly the greedy traceback path from src to snk, else an error code."""
    a, b, t = _u8(a), _u8(b), sch.table()
    o = ops.encode()
    return int(_L().orc_verify_path(_ptr(a), len(a), _ptr(b), len(b), _ptr(t), sch.alphabet,
                                    sch.gap_open, sch.gap_extend, src, snk, o, len(o)))


def local_matrix(a, b, sch: Scheme = DNA) -> np.ndarray:
    a, b, t = _u8(a), _u8(b), sch.table()
    out = np.zeros((len(a) + 1, len(b) + 1), dtype=np.int64)
    _L().orc_local_matrix(_ptr(a), len(a), _ptr(b), len(b), _ptr(t), sch.alphabet,
                          sch.gap_open, sch.gap_extend, _ptr(out))
    return out


def ops_to_cigar(ops: str, a_sub, b_sub) -> str:
    """'M' ops become '=' (identical codes) or 'X'; runs are length-prefixed."""
    a_sub, b_sub = _u8(a_sub), _u8(b_sub)
    out, i, j = [], 0, 0
    for o in ops:
        if o == "M":
            out.append("=" if a_sub[i] == b_sub[j] else "X")
            i += 1
            j += 1
        elif o == "I":
            out.append("I")
            i += 1
        else:
            out.append("D")
            j += 1
    res, k = [], 0
    while k < len(out):
        r = k
        while r < len(out) and out[r] == out[k]:
            r += 1
        res.append(f"{r - k}{out[k]}")
        k = r
    return "".join(res)


def cigar_to_ops(cigar: str) -> str:
    ops, num = [], ""
    for ch in cigar:
        if ch.isdigit():
            num += ch
        else:
            ops.append(("M" if ch in "=X" else ch) * int(num))
            num = ""
    return "".join(ops)


@dataclass
class Alignment:
    score: int
    a_begin: int
    a_end: int
    b_begin: int
    b_end: int
    cigar: str


def align(a, b, sch: Scheme = DNA) -> Alignment:
    """Full oracle pipeline: score + end point, start point, canonical alignment."""
    a, b = _u8(a), _u8(b)
    S, ei, ej = local_score(a, b, sch)
    if S == 0:
        return Alignment(0, -1, -1, -1, -1, "")
    bi, bj, _ = reverse_start(a, b, ei, ej, S, sch)
    v, ops = global_trace(a[bi:ei], b[bj:ej], sch)
    if v != S:
        raise AssertionError(f"global value {v} != local score {S}")
    return Alignment(S, bi, ei, bj, ej, ops_to_cigar(ops, a[bi:ei], b[bj:ej]))
