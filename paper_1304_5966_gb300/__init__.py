"""Python binding of libswgb (include/swgb.h): argument marshalling only.

Exact affine-gap Smith-Waterman on one GB300 (sm_103a): score and end point,
start point and the canonical alignment (Korpar & Sikic, SW#, Sec. 2).  Every
step runs in the library's CUDA kernels; this module only converts arguments.
PyTorch supplies the device workspace and the CUDA stream.

    import paper_1304_5966_gb300 as sw
    ctx = sw.sw_ctx_create(workspace_bytes=1 << 30)
    r = sw.sw_score(ctx, a, b)          # a, b: uint8 codes (numpy = host, torch cuda = device)
    r = sw.sw_align(ctx, a, b)          # r.score, r.a_begin, ..., r.cigar

There is no CPU fallback: if the shared library has not been built (see
``build.py``) importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libswgb.so")

SW_OK, SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT, SW_EBUSY, SW_ENOTIMPL, SW_EPENDING = range(8)
SW_FLAG_DEVICE_INPUT = 0x1
SW_FLAG_SCORE_ONLY = 0x2
SW_FLAG_NO_PRUNE = 0x4
SW_FLAG_FORCE_INT32 = 0x8
SW_FLAG_FORCE_INT16 = 0x10
SW_FLAG_BOTH_STRANDS = 0x20
SW_OPT_ROWS_PER_THREAD, SW_OPT_WARPS_PER_SM, SW_OPT_TIMEOUT_MS, SW_OPT_FAULT_BAND, \
    SW_OPT_CKPT_BANDS, SW_OPT_LEAF_CELLS, SW_OPT_FORWARD_LANES, SW_OPT_TRACE, SW_OPT_AUTOTUNE = range(1, 10)


class SwError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class _Scheme(ctypes.Structure):
    _fields_ = [("alphabet", ctypes.c_int32), ("matrix", ctypes.c_void_p),
                ("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("cells", ctypes.c_int64), ("cells_computed", ctypes.c_int64),
                ("tiles_total", ctypes.c_int64), ("tiles_pruned", ctypes.c_int64),
                ("int16_reruns", ctypes.c_int32), ("levels", ctypes.c_int32),
                ("ms_forward", ctypes.c_float), ("ms_start", ctypes.c_float),
                ("ms_align", ctypes.c_float), ("fwd_cells", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("start_cells", ctypes.c_int64),
                ("align_cells", ctypes.c_int64), ("band_rows", ctypes.c_int32), ("tuned", ctypes.c_int32),
                ("cta_warps", ctypes.c_int32)]


class _Result(ctypes.Structure):
    _fields_ = [("score", ctypes.c_int64), ("a_begin", ctypes.c_int64), ("a_end", ctypes.c_int64),
                ("b_begin", ctypes.c_int64), ("b_end", ctypes.c_int64),
                ("cigar", ctypes.c_void_p), ("cigar_len", ctypes.c_int64), ("stats", _Stats),
                ("strand", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# numpy view of a _Result array (same layout): score, coordinates, the CIGAR
# pointer and the per-pair cell count, read in bulk for large batches
_RESULT_DTYPE = np.dtype({"names": ["score", "a_begin", "a_end", "b_begin", "b_end", "cigar", "cells", "strand"],
                          "formats": ["<i8"] * 5 + ["<u8", "<i8", "<i4"],
                          "offsets": [_Result.score.offset, _Result.a_begin.offset, _Result.a_end.offset,
                                      _Result.b_begin.offset, _Result.b_end.offset, _Result.cigar.offset,
                                      _Result.stats.offset + _Stats.cells.offset, _Result.strand.offset],
                          "itemsize": ctypes.sizeof(_Result)})


class _Pair(ctypes.Structure):
    _fields_ = [("a", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("b", ctypes.c_void_p), ("m", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libswgb; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libswgb not built ({_LIB_PATH}); run paper_1304_5966_gb300/build.py")
        L = ctypes.CDLL(_LIB_PATH)
        P, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        L.sw_ctx_create.argtypes = [ctypes.c_int, P, P, ctypes.c_uint64, ctypes.POINTER(P)]
        L.sw_ctx_destroy.argtypes = [P]
        L.sw_ctx_destroy.restype = None
        L.sw_ctx_last_error.argtypes = [P]
        L.sw_ctx_last_error.restype = ctypes.c_char_p
        L.sw_strerror.argtypes = [ctypes.c_int]
        L.sw_strerror.restype = ctypes.c_char_p
        L.sw_ctx_set_option.argtypes = [P, ctypes.c_int, i64]
        L.sw_ctx_tuning_export.argtypes = [P, ctypes.c_char_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.sw_ctx_tuning_import.argtypes = [P, ctypes.c_char_p]
        for fn in ("sw_score", "sw_align", "sw_score_plain"):
            getattr(L, fn).argtypes = [P, P, i64, P, i64, ctypes.POINTER(_Scheme), i32,
                                       ctypes.POINTER(_Result)]
        L.sw_align_batch.argtypes = [P, ctypes.POINTER(_Pair), i32, ctypes.POINTER(_Scheme), i32,
                                     ctypes.POINTER(_Result)]
        L.sw_score_static.argtypes = [P, i64, P, i64, ctypes.POINTER(_Scheme), P, ctypes.POINTER(_Result)]
        L.sw_score_job_create.argtypes = [P, P, i64, P, i64, ctypes.POINTER(_Scheme), i32, ctypes.POINTER(P)]
        L.sw_score_job_run.argtypes = [P, i64, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.sw_score_job_snapshot.argtypes = [P, P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
        L.sw_score_job_resume.argtypes = [P, P, i64, P, i64, ctypes.POINTER(_Scheme), i32, P, ctypes.c_uint64,
                                          ctypes.POINTER(P)]
        L.sw_score_job_result.argtypes = [P, ctypes.POINTER(_Result)]
        L.sw_score_job_destroy.argtypes = [P]
        L.sw_score_job_destroy.restype = None
        L.sw_server_create.argtypes = [P, i32, ctypes.c_uint64, ctypes.POINTER(P)]
        L.sw_server_submit.argtypes = [P, P, i64, P, i64, ctypes.POINTER(_Scheme), i32,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.sw_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(_Result), i64]
        L.sw_server_cancel.argtypes = [P, ctypes.c_uint64]
        L.sw_server_destroy.argtypes = [P]
        L.sw_server_destroy.restype = None
        L.sw_result_free.argtypes = [ctypes.POINTER(_Result)]
        L.sw_result_free.restype = None
        _lib = L
    return _lib


@dataclass
class Scheme:
    """Substitution scores and affine gap costs (gap of length k = go + ge*(k-1))."""
    match: int = 1
    mismatch: int = -3
    gap_open: int = 5
    gap_extend: int = 2
    alphabet: int = 4
    matrix: tuple | None = None

    def _c(self):
        s = _Scheme(self.alphabet, None, self.match, self.mismatch, self.gap_open, self.gap_extend)
        keep = None
        if self.matrix is not None:
            keep = np.ascontiguousarray(np.asarray(self.matrix, dtype=np.int8))
            s.matrix = keep.ctypes.data
        return s, keep


DNA = Scheme()


@dataclass
class Result:
    score: int
    a_begin: int
    a_end: int
    b_begin: int
    b_end: int
    cigar: str | None
    stats: dict = field(default_factory=dict)
    strand: int = 0          # 1: the reverse complement of B (SW_FLAG_BOTH_STRANDS)


class Context:
    """A library context: device, CUDA stream and a device workspace from torch."""

    def __init__(self, device: int = 0, workspace_bytes: int = 1 << 30, stream=None, workspace=None):
        import torch
        self.device = device
        torch.cuda.set_device(device)
        if workspace is None:
            workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=f"cuda:{device}")
        self.workspace = workspace            # kept alive for the context's lifetime
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        st = lib().sw_ctx_create(device, ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.c_void_p(workspace.data_ptr()),
                                 workspace.numel() * workspace.element_size(), ctypes.byref(h))
        if st != SW_OK:
            raise SwError(st, "sw_ctx_create failed: " + lib().sw_strerror(st).decode())
        self.handle = h

    def set_option(self, option: int, value: int):
        _check(self, lib().sw_ctx_set_option(self.handle, option, int(value)))

    def tuning_export(self) -> str:
        """The batch autotuner's table (batch shape -> band height) as text."""
        n = ctypes.c_uint64()
        st = lib().sw_ctx_tuning_export(self.handle, None, 0, ctypes.byref(n))
        if st not in (SW_OK, SW_ENOMEM):
            _check(self, st)
        buf = ctypes.create_string_buffer(n.value + 1)
        _check(self, lib().sw_ctx_tuning_export(self.handle, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def tuning_import(self, text: str):
        """Merge a table written by tuning_export on the same GPU model."""
        _check(self, lib().sw_ctx_tuning_import(self.handle, text.encode()))

    def close(self):
        if getattr(self, "handle", None):
            lib().sw_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().sw_ctx_last_error(self.handle).decode()


def sw_ctx_create(device: int = 0, workspace_bytes: int = 1 << 30, stream=None, workspace=None) -> Context:
    return Context(device, workspace_bytes, stream, workspace)


def sw_ctx_destroy(ctx: Context):
    ctx.close()


def _check(ctx, st):
    if st != SW_OK:
        raise SwError(st, f"{lib().sw_strerror(st).decode()}: {ctx.last_error()}")


def _seq(x):
    """(pointer, length, is_device, keepalive) for a numpy/bytes/torch sequence of codes."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.uint8 or not x.is_contiguous():
                raise TypeError("device sequences must be contiguous torch.uint8")
            return x.data_ptr(), x.numel(), x.is_cuda, x
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(x, dtype=np.uint8))
    return arr.ctypes.data, len(arr), False, arr


def _result(r: _Result) -> Result:
    cig = None
    if r.cigar:
        cig = ctypes.string_at(r.cigar, r.cigar_len).decode()
    st = {f: getattr(r.stats, f) for f, _ in _Stats._fields_}
    return Result(int(r.score), int(r.a_begin), int(r.a_end), int(r.b_begin), int(r.b_end), cig, st,
                  int(r.strand))


def _pairwise(fn, ctx, a, b, scheme, flags):
    pa, n, da, ka = _seq(a)
    pb, m, db, kb = _seq(b)
    if da != db:
        raise ValueError("a and b must both be host or both be device sequences")
    if da:
        flags |= SW_FLAG_DEVICE_INPUT
    sch, keep = (scheme or DNA)._c()
    res = _Result()
    st = fn(ctx.handle, pa, n, pb, m, ctypes.byref(sch), flags, ctypes.byref(res))
    _check(ctx, st)
    out = _result(res)
    lib().sw_result_free(ctypes.byref(res))
    return out


def sw_score(ctx: Context, a, b, scheme: Scheme | None = None, flags: int = 0) -> Result:
    """Best local score and end point (Sec. 2, forward pass with pruning)."""
    return _pairwise(lib().sw_score, ctx, a, b, scheme, flags)


def sw_align(ctx: Context, a, b, scheme: Scheme | None = None, flags: int = 0) -> Result:
    """Score, start/end point and canonical CIGAR (Sec. 2, all three phases)."""
    return _pairwise(lib().sw_align, ctx, a, b, scheme, flags)


def sw_score_plain(ctx: Context, a, b, scheme: Scheme | None = None, flags: int = 0) -> Result:
    """The plain anti-diagonal GPU baseline (one thread per cell, one launch per diagonal)."""
    return _pairwise(lib().sw_score_plain, ctx, a, b, scheme, flags)


def _host_pairs(pairs):
    """sw_pair records of host numpy uint8 pairs as one int64 array (the fast
    path for large batches), or None when any sequence is something else."""
    u8 = np.dtype(np.uint8)
    rows = []
    for a, b in pairs:
        if (a.__class__ is not np.ndarray or b.__class__ is not np.ndarray or a.dtype != u8 or b.dtype != u8
                or not a.flags.c_contiguous or not b.flags.c_contiguous):
            return None
        rows.append((a.ctypes.data, a.size, b.ctypes.data, b.size))
    return np.array(rows, dtype=np.int64).reshape(len(rows), 4)


def sw_align_batch(ctx: Context, pairs, scheme: Scheme | None = None, flags: int = 0):
    """Many pairs in one persistent launch; returns one Result per pair, in order.
    With SW_FLAG_BOTH_STRANDS each pair is also run against the reverse
    complement of B and the better strand kept (Result.strand)."""
    keep = []
    dev = None
    packed = _host_pairs(pairs) if len(pairs) else None
    if packed is not None:
        keep.append(packed)
        cp = packed.ctypes.data_as(ctypes.POINTER(_Pair))
    else:
        cp = (_Pair * max(1, len(pairs)))()
        for k, (a, b) in enumerate(pairs):
            pa, n, da, ka = _seq(a)
            pb, m, db, kb = _seq(b)
            if da != db or (dev is not None and dev != da):
                raise ValueError("all sequences must be host, or all device")
            dev = da
            keep += [ka, kb]
            cp[k] = _Pair(pa, n, pb, m)
    if dev:
        flags |= SW_FLAG_DEVICE_INPUT
    sch, kk = (scheme or DNA)._c()
    outs = (_Result * max(1, len(pairs)))()
    st = lib().sw_align_batch(ctx.handle, cp, len(pairs), ctypes.byref(sch), flags, outs)
    _check(ctx, st)
    return _batch_results(outs, len(pairs))


def _batch_results(outs, count: int):
    """Results of a batch call: the call's statistics are in the first result
    (every later one carries its cell count only); read through one array view."""
    if count == 0:
        return []
    view = np.frombuffer((ctypes.c_char * (ctypes.sizeof(_Result) * count)).from_buffer(outs),
                         dtype=_RESULT_DTYPE, count=count)
    score, a0, a1 = view["score"].tolist(), view["a_begin"].tolist(), view["a_end"].tolist()
    b0, b1, cells = view["b_begin"].tolist(), view["b_end"].tolist(), view["cells"].tolist()
    strand = view["strand"].tolist()
    has_cigar = view["cigar"].any()
    res = []
    for k in range(count):
        cig = None
        if has_cigar and outs[k].cigar:
            cig = ctypes.string_at(outs[k].cigar, outs[k].cigar_len).decode()
            lib().sw_result_free(ctypes.byref(outs[k]))
        st = {f: getattr(outs[0].stats, f) for f, _ in _Stats._fields_} if k == 0 else {"cells": cells[k]}
        res.append(Result(score[k], a0[k], a1[k], b0[k], b1[k], cig, st, strand[k]))
    return res


def sw_score_static(a, b, scheme: Scheme | None = None, stream=None) -> Result:
    """Score and end point without any device allocation (library-wide static
    scratch; device inputs only; n <= 16,777,216, m <= 1,048,576).  For callers
    that cannot allocate device memory at call time.  Calls must not overlap."""
    import torch
    pa, n, da, ka = _seq(a)
    pb, m, db, kb = _seq(b)
    if not (da and db):
        raise ValueError("sw_score_static takes device sequences")
    s = stream if stream is not None else torch.cuda.current_stream()
    sch, keep = (scheme or DNA)._c()
    res = _Result()
    st = lib().sw_score_static(pa, n, pb, m, ctypes.byref(sch), ctypes.c_void_p(s.cuda_stream), ctypes.byref(res))
    if st != SW_OK:
        raise SwError(st, f"sw_score_static: {lib().sw_strerror(st).decode()}")
    return _result(res)


class ScoreJob:
    """A score pass run in segments of row bands, whose state can be saved to
    host memory (snapshot) and resumed (sw_score_job_resume)."""

    def __init__(self, ctx: Context, handle, keep):
        self.ctx, self.handle, self._keep = ctx, handle, keep
        self.bands_done, self.bands_total, self.wave_bands = 0, None, None
        self.run(0)

    def run(self, bands: int = -1):
        """Run up to `bands` more bands (-1: all that are left, 0: none);
        returns (bands done, bands in total).  `wave_bands` is how many bands
        the GPU runs at once: segments of whole waves add the least time."""
        d, t, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(self.ctx, lib().sw_score_job_run(self.handle, int(bands), ctypes.byref(d), ctypes.byref(t),
                                                ctypes.byref(w)))
        self.bands_done, self.bands_total, self.wave_bands = d.value, t.value, w.value
        return d.value, t.value

    def snapshot(self) -> bytes:
        n = ctypes.c_uint64()
        st = lib().sw_score_job_snapshot(self.handle, None, 0, ctypes.byref(n))
        if st not in (SW_OK, SW_ENOMEM):
            _check(self.ctx, st)
        buf = ctypes.create_string_buffer(n.value)
        _check(self.ctx, lib().sw_score_job_snapshot(self.handle, buf, n.value, ctypes.byref(n)))
        return buf.raw[:n.value]

    def result(self) -> Result:
        res = _Result()
        _check(self.ctx, lib().sw_score_job_result(self.handle, ctypes.byref(res)))
        return _result(res)

    def close(self):
        if getattr(self, "handle", None):
            lib().sw_score_job_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _job_args(a, b, scheme, flags):
    pa, n, da, ka = _seq(a)
    pb, m, db, kb = _seq(b)
    if da != db:
        raise ValueError("a and b must both be host or both be device sequences")
    if da:
        flags |= SW_FLAG_DEVICE_INPUT
    sch, keep = (scheme or DNA)._c()
    return pa, n, pb, m, sch, flags, (ka, kb, keep)


def sw_score_job_create(ctx: Context, a, b, scheme: Scheme | None = None, flags: int = 0) -> ScoreJob:
    """A checkpointable score pass over (a, b); run it with ScoreJob.run."""
    pa, n, pb, m, sch, flags, keep = _job_args(a, b, scheme, flags)
    h = ctypes.c_void_p()
    _check(ctx, lib().sw_score_job_create(ctx.handle, pa, n, pb, m, ctypes.byref(sch), flags, ctypes.byref(h)))
    return ScoreJob(ctx, h, keep)


def sw_score_job_resume(ctx: Context, a, b, snapshot: bytes, scheme: Scheme | None = None,
                        flags: int = 0) -> ScoreJob:
    """Rebuild a job from ScoreJob.snapshot() for the same sequences, scheme and flags."""
    pa, n, pb, m, sch, flags, keep = _job_args(a, b, scheme, flags)
    h = ctypes.c_void_p()
    snap = ctypes.create_string_buffer(bytes(snapshot), len(snapshot))
    _check(ctx, lib().sw_score_job_resume(ctx.handle, pa, n, pb, m, ctypes.byref(sch), flags, snap,
                                          len(snapshot), ctypes.byref(h)))
    return ScoreJob(ctx, h, keep)


class Server:
    """Continuous-batching request server (sw_server_*).  submit() copies the
    host sequences and returns a ticket; poll() waits for the result."""

    def __init__(self, ctx: Context, workers: int = 4, device_budget: int = 0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        st = lib().sw_server_create(ctx.handle, workers, device_budget, ctypes.byref(h))
        if st != SW_OK:
            raise SwError(st, "sw_server_create failed")
        self.handle = h

    def submit(self, a, b, scheme: Scheme | None = None, score_only: bool = False, flags: int = 0) -> int:
        pa, n, da, ka = _seq(a)
        pb, m, db, kb = _seq(b)
        if da or db:
            raise ValueError("server requests take host sequences")
        sch, keep = (scheme or DNA)._c()
        t = ctypes.c_uint64()
        st = lib().sw_server_submit(self.handle, pa, n, pb, m, ctypes.byref(sch),
                                    flags | (SW_FLAG_SCORE_ONLY if score_only else 0), ctypes.byref(t))
        if st != SW_OK:
            raise SwError(st, f"sw_server_submit: {lib().sw_strerror(st).decode()}")
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = -1):
        """The Result, or None while the request is pending."""
        res = _Result()
        st = lib().sw_server_poll(self.handle, ticket, ctypes.byref(res), timeout_us)
        if st == SW_EPENDING:
            return None
        out = _result(res)
        lib().sw_result_free(ctypes.byref(res))
        if st != SW_OK:
            raise SwError(st, f"request {ticket}: {lib().sw_strerror(st).decode()}")
        return out

    def cancel(self, ticket: int) -> int:
        return lib().sw_server_cancel(self.handle, ticket)

    def close(self):
        if getattr(self, "handle", None):
            lib().sw_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sw_server_create(ctx: Context, workers: int = 4, device_budget: int = 0) -> Server:
    return Server(ctx, workers, device_budget)
