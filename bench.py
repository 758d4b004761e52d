"""Benchmark: exact affine-gap Smith-Waterman on one GB300 (sm_103a).

One step = the whole hot path on the chromosome-scale pair: forward score pass
with end point (pruned), reverse start-point pass and linear-space
reconstruction of the CIGAR (sw_align), on the 5,000,000 x ~4,950,000 synthetic
DNA pair (GC 41 %, tandem repeats, 10 % substitutions, 1 % indels, a 20 kbp
inversion and a 50 kbp deletion).  Metric: GCUPS = n*m / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is timed with inputs resident in HBM (CUDA
events on the library's stream; L2 flushed before every step by writing a
256 MiB buffer); `e2e` is the same call with host (pinned) buffers, the
host->device copies and the CIGAR read-back inside the timed region.
`roofline` is for the forward-pass kernel (the dominant one): computed cells
x 3.5 integer ops per cell (the minimal DPX cell update: 7 ops per int16x2 cell pair)
per second, against the
integer pipe's lane rate (64 lane-ops / clock / SM, measured) x SMs x the SM
clock sampled during the run.  `cpu_baseline` is the CPU oracle (oracle/) on a
bounded prefix sample of the same pair.  `--impl reference` times that oracle
alone (there is no runnable reference implementation of the paper).

With N > 1 (torchrun), every rank aligns its own copy of the pair (replicas
only: the single-pair path does not shard) and value = total cells / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

OPS_PER_CELL = 3.5        # minimal cell update on int16x2 DPX lanes: 7 ops per two cells
INT_LANES_PER_CLK = 64    # measured: DPX (32- and 16x2-bit) / PRMT lane ops per clock per SM
SAMPLE_EDGE = 40_000      # CPU oracle sample: the first 40k x 40k of the pair
# DRAM bytes (read + write) of one forward launch of this step, from one ncu
# capture of the timed step's forward pass (profiles/fwd16_kernel_dram_pair_5m_bench.md);
# set to None whenever the forward kernel changes
FWD_TRAFFIC_BYTES = 329_223_936 + 3_348_415_488


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-extras", action="store_true", help="skip the batch / plain comparisons")
    p.add_argument("--workload", default="pair_5m", choices=["pair_5m", "score_500k", "score_2m", "score_5m_1m"],
                   help="score_500k / score_2m / score_5m_1m: forward pass alone on a 500 kbp pair, a 2 Mbp x "
                        "1 Mbp homologous pair, or the first 5,000,000 x 1,000,000 of the bench pair (the bench's "
                        "band height) -- profiling cases")
    p.add_argument("--workspace-gb", type=int, default=0, help="device workspace (default by workload)")
    return p.parse_args()


def run_profile_case(args):
    """Cases for ncu: sw_score on a 500,000 x ~500,000 homologous pair (score_500k),
    on the first 2,000,000 x 1,000,000 of a homologous pair (score_2m, enough
    bands and columns to fill the band pipeline) or on the first 5,000,000 x
    1,000,000 of the bench pair (score_5m_1m: the bench's 1,024-row bands)."""
    import torch
    import paper_1304_5966_gb300 as sw
    from gen import synth
    if args.workload == "score_5m_1m":
        a, b = synth.pair_5m()
        b = b[:1_000_000].copy()
    elif args.workload == "score_2m":
        a, b = synth.pair_homologous(2_000_000, seed=13, gc_permille=410)
        b = b[:1_000_000].copy()
    else:
        a, b = synth.pair_homologous(500_000, seed=13, gc_permille=410)
    ctx = sw.sw_ctx_create(0, workspace_bytes=(args.workspace_gb or 1) << 30)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    for _ in range(args.warmup):
        sw.sw_score(ctx, ta, tb)
    ms = []
    for _ in range(args.steps):
        r = sw.sw_score(ctx, ta, tb)
        ms.append(r.stats["ms_forward"])
    print(json.dumps({"workload": args.workload, "n": len(a), "m": len(b), "score": r.score,
                      "end": [r.a_end, r.b_end], "ms_forward": ms,
                      "gcups": round(len(a) * len(b) / statistics.mean(ms) / 1e6, 1),
                      "fwd_cells": r.stats["fwd_cells"], "tiles_pruned": r.stats["tiles_pruned"],
                      "tiles_total": r.stats["tiles_total"]}), flush=True)


def _config(n: int, m: int, world: int) -> dict:
    """The workload both arms report (ours and the oracle's)."""
    return {"workload": f"pair_5m: {n} x {m} DNA pair (GC 41%, tandem repeats, 10% subst, 1% ins, "
                        f"1% del, 20 kbp inversion, 50 kbp deletion); sw_align = score + end, "
                        f"start, CIGAR; match +1, mismatch -3, gap 5 + 2(k-1)",
            "l2": "flushed before every step (256 MiB write); step working set < L2",
            "arithmetic": "exact integer scores: forward and start passes on int16x2 DPX lanes with "
                          "per-warp offsets, int32 boundary rows and reconstruction",
            "parallelism": f"replicas x{world}"}


def _max_over_ranks(dist, x: float, device: str) -> float:
    """The largest x over all ranks (every rank gets it); x itself without a
    process group.  The job's time is the slowest replica's."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_gcups(world: int, cells: int, steps: int, total_s: float) -> float:
    """Whole-job GCUPS: every replica aligns the pair `steps` times."""
    return world * cells * steps / total_s / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{gpu}.csv")
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.strip().split(", ") for l in open(self.path) if l.strip()]
        except OSError:
            return out
        mhz = [int(r[0].split()[0]) for r in rows if r and r[0].split()[0].isdigit()]
        mx = [int(r[1].split()[0]) for r in rows if len(r) > 1 and r[1].split()[0].isdigit()]
        if mhz:
            out["sm_mhz"] = statistics.median(mhz)
            out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].strip() == "Active":
                    seen.add(nm)
        out["reasons"] = sorted(seen)
        out["samples"] = len(mhz)
        return out


def cpu_baseline(a, b):
    """The oracle as it stands, single thread, on the first SAMPLE_EDGE^2 cells."""
    import oracle
    oracle.build()
    sa, sb = a[:SAMPLE_EDGE], b[:SAMPLE_EDGE]
    t = time.perf_counter()
    r = oracle.align(sa, sb)
    dt = time.perf_counter() - t
    cells = len(sa) * len(sb)
    return {"value": round(cells / dt / 1e9, 4), "unit": "GCUPS", "cores": 1, "kind": "oracle",
            "sample": f"oracle.align (score, start, traceback) on the first {len(sa)} x {len(sb)} "
                      f"bases of the pair, {dt:.1f} s, score {r.score}"}


def run_reference(args):
    ws, rank, _ = _dist()
    from gen import synth
    a, b = synth.pair_5m()
    if rank != 0:
        return
    vals = []
    for _ in range(args.warmup):
        pass      # the oracle has no warm-up state; steps below are each a full sample
    for _ in range(args.steps):
        cb = cpu_baseline(a, b)
        vals.append(cb["value"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "GCUPS", "value": v, "unit": "GCUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": _config(len(a), len(b), args.gpus),
            "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batch(sw, ctx, reps: int = 3):
    """4,096 pairs (lengths log-uniform 100..20,000 per side): one batched call vs
    the single-pair path (sw_score per pair) and the plain anti-diagonal path."""
    import torch
    from gen import synth
    pairs = synth.batch_pairs()
    cells = sum(len(a) * len(b) for a, b in pairs)
    sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY)          # warm-up
    ts, st = [], None
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = sw.sw_align_batch(ctx, pairs, flags=sw.SW_FLAG_SCORE_ONLY)
        ts.append(time.perf_counter() - t0)
        st = res[0].stats
    batch_s = min(ts)
    # single-pair path and plain path on a seeded sample of the same pairs
    sample = pairs[::16]
    scells = sum(len(a) * len(b) for a, b in sample)
    t0 = time.perf_counter()
    for a, b in sample:
        sw.sw_score(ctx, a, b)
    single_s = time.perf_counter() - t0
    psample = pairs[::256]
    pcells = sum(len(a) * len(b) for a, b in psample)
    t0 = time.perf_counter()
    for a, b in psample:
        sw.sw_score_plain(ctx, a, b)
    plain_s = time.perf_counter() - t0
    g = cells / batch_s / 1e9
    both = bench_both_strands(sw, ctx, pairs, cells, res)
    return {"pairs": len(pairs), "cells": cells, "ms": round(batch_s * 1e3, 2), "gcups": round(g, 1),
            "both_strands": both,
            "kernel_ms": round(st["ms_forward"], 2), "int16_reruns": st["int16_reruns"],
            "single_pair_path_gcups": round(scells / single_s / 1e9, 1),
            "plain_path_gcups": round(pcells / plain_s / 1e9, 2),
            "vs_single_pair_path": round(g / (scells / single_s / 1e9), 2),
            "vs_plain_path": round(g / (pcells / plain_s / 1e9), 1),
            "note": "wall time of the score-only batch call incl. H2D of the packed pairs; "
                    "single-pair path timed on every 16th pair, plain path on every 256th"}


def bench_both_strands(sw, ctx, pairs, cells, one_strand, reps: int = 3):
    """The same batch against both strands of B (SW_FLAG_BOTH_STRANDS): wall
    time, GCUPS over the cells of both strands, and the forward-strand results
    kept wherever they win."""
    try:
        fl = sw.SW_FLAG_SCORE_ONLY | sw.SW_FLAG_BOTH_STRANDS
        sw.sw_align_batch(ctx, pairs, flags=fl)                       # warm-up (tunes the doubled shape)
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            res = sw.sw_align_batch(ctx, pairs, flags=fl)
            ts.append(time.perf_counter() - t0)
        t = min(ts)
        fwd_kept = all((r.score, r.a_end, r.b_end) == (o.score, o.a_end, o.b_end)
                       for r, o in zip(res, one_strand) if r.strand == 0)
        return {"ms": round(t * 1e3, 2), "gcups": round(2 * cells / t / 1e9, 1),
                "reverse_wins": sum(r.strand for r in res), "forward_results_unchanged": fwd_kept}
    except Exception as e:          # a side measurement never takes the bench line down
        return {"error": str(e)}


def bench_checkpointed(sw, ctx, ta, tb, one_pass):
    """The pruned score pass as a checkpointed job: segments of one wave of
    bands, a host snapshot after each; same score and end point as one pass."""
    try:
        t0 = time.perf_counter()
        job = sw.sw_score_job_create(ctx, ta, tb)
        snap_bytes, segs = 0, 0
        while True:
            jdone, jtotal = job.run(job.wave_bands)
            snap_bytes = len(job.snapshot())
            segs += 1
            if jdone == jtotal:
                break
        rj = job.result()
        job.close()
        job_s = time.perf_counter() - t0
    except Exception as e:          # a side measurement never takes the bench line down
        return {"error": str(e)}
    return {"segments": segs, "bands": jtotal, "wave_bands": job.wave_bands,
            "snapshot_mb": round(snap_bytes / 2 ** 20, 1), "wall_s": round(job_s, 2),
            "kernel_ms": round(rj.stats["ms_forward"], 1),
            "vs_one_pass_kernel": round(rj.stats["ms_forward"] / one_pass.stats["ms_forward"], 3),
            "same_score_and_end": (rj.score, rj.a_end, rj.b_end) == (one_pass.score, one_pass.a_end, one_pass.b_end)}


def bench_small_pairs(sw, ctx, reps: int = 9):
    """The 1,000 x ~1,000 pair (an 800-base mutated window of A in random
    flanks) and the 100,000 x ~100,000 homologous pair with tandem repeats:
    median wall latency of sw_align and of sw_score per call (host inputs,
    results read back), and their GCUPS."""
    from gen import synth
    out = {}
    for name, (a, b) in (("pair_1k", synth.pair_1k()), ("pair_100k", synth.pair_100k())):
        row = {"n": len(a), "m": len(b)}
        for fn in ("sw_score", "sw_align"):
            f = getattr(sw, fn)
            f(ctx, a, b)                                   # warm-up
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                r = f(ctx, a, b)
                ts.append(time.perf_counter() - t0)
            t = statistics.median(ts)
            row[fn] = {"ms": round(t * 1e3, 3), "gcups": round(len(a) * len(b) / t / 1e9, 1), "score": r.score}
        out[name] = row
    return out


def bench_serving(sw, ctx, rates=(10.0, 100.0, 1000.0), count: int = 40):
    """Poisson arrivals of pairs with L log-uniform in [1e3, 1e6] (70 % score-only,
    30 % alignment), submitted at their arrival times to a 4-worker server."""
    import threading
    from gen import synth
    out = []
    for rate in rates:
        stream = synth.serve_stream(count, rate, seed=5)
        srv = sw.Server(ctx, workers=4, device_budget=16 << 30)
        sub, done = {}, {}
        tickets = [None] * count
        t_start = time.perf_counter()

        def producer():
            for k, (t_arr, a, b, align) in enumerate(stream):
                dt = t_start + t_arr - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                sub[k] = time.perf_counter()
                tickets[k] = srv.submit(a, b, score_only=not align)

        th = threading.Thread(target=producer)
        th.start()
        pending = set(range(count))
        while pending:
            for k in list(pending):
                if tickets[k] is None:
                    continue
                r = srv.poll(tickets[k], timeout_us=0)
                if r is not None:
                    done[k] = time.perf_counter()
                    pending.discard(k)
            time.sleep(0.0005)
        th.join()
        srv.close()
        lat = sorted(done[k] - sub[k] for k in range(count))
        span = max(done.values()) - min(sub.values())
        cells = sum(len(a) * len(b) for _, a, b, _ in stream)
        out.append({"offered_rps": rate, "requests": count,
                    "p50_ms": round(1e3 * lat[len(lat) // 2], 1),
                    "p99_ms": round(1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], 1),
                    "achieved_rps": round(count / span, 2), "sustained_gcups": round(cells / span / 1e9, 1)})
    return out


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("score_500k", "score_2m", "score_5m_1m"):
        return run_profile_case(args)
    ws, rank, local = _dist()
    import numpy as np
    import torch
    import paper_1304_5966_gb300 as sw
    from gen import synth

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    a, b = synth.pair_5m()
    n, m = len(a), len(b)
    ctx = sw.sw_ctx_create(local, workspace_bytes=(args.workspace_gb or 24) << 30)
    stream = ctx.stream
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(dev=True):
        if dev:
            return sw.sw_align(ctx, ta, tb)
        return sw.sw_align(ctx, ha, hb)

    for _ in range(args.warmup):
        r = step()
    ha = torch.from_numpy(a).pin_memory()
    hb = torch.from_numpy(b).pin_memory()

    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, fwd_ms, fwd_cells, launches = [], [], [], 0
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        ev0.record(stream)
        r = step()
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
        fwd_ms.append(r.stats["ms_forward"])
        fwd_cells.append(r.stats["fwd_cells"])
        launches += r.stats["kernel_launches"]
    torch.cuda.synchronize()
    clk = clocks.stop()
    total = _max_over_ranks(dist, sum(times), "cuda")
    if dist:
        dist.barrier()

    # end to end through the public API: host buffers in, CIGAR back on the host
    e2e_times = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        re = step(dev=False)
        e2e_times.append(time.perf_counter() - t0)
    assert (re.score, re.cigar) == (r.score, r.cigar)
    e2e_total = _max_over_ranks(dist, sum(e2e_times), "cuda")

    extras = {}
    if not args.no_extras and rank == 0:
        # score-only forward pass, pruning on and off (same score and end point)
        rs = sw.sw_score(ctx, ta, tb)
        rn = sw.sw_score(ctx, ta, tb, flags=sw.SW_FLAG_NO_PRUNE)
        assert (rs.score, rs.a_end, rs.b_end) == (rn.score, rn.a_end, rn.b_end) == (r.score, r.a_end, r.b_end)
        extras["score_pass"] = {
            "gcups_pruned": round(n * m / rs.stats["ms_forward"] / 1e6, 1),
            "gcups_unpruned": round(n * m / rn.stats["ms_forward"] / 1e6, 1),
            "ms_pruned": round(rs.stats["ms_forward"], 1), "ms_unpruned": round(rn.stats["ms_forward"], 1),
            "tiles_pruned_frac": round(rs.stats["tiles_pruned"] / max(1, rs.stats["tiles_total"]), 4),
            "roofline_frac_unpruned": round(rn.stats["fwd_cells"] * OPS_PER_CELL / (rn.stats["ms_forward"] / 1e3) /
                                            (torch.cuda.get_device_properties(local).multi_processor_count *
                                             INT_LANES_PER_CLK * (clk["sm_mhz"] or 2070) * 1e6), 4)}
        extras["checkpointed_score_pass"] = bench_checkpointed(sw, ctx, ta, tb, rs)
        # the plain GPU path (one thread per cell, one launch per anti-diagonal)
        ps = 20_000
        rp = sw.sw_score_plain(ctx, a[:ps], b[:ps])
        rq = sw.sw_score(ctx, a[:ps], b[:ps])
        assert (rp.score, rp.a_end, rp.b_end) == (rq.score, rq.a_end, rq.b_end)
        extras["plain_path"] = {"sample": f"{ps} x {ps} prefix", "gcups": round(ps * ps / rp.stats["ms_forward"] / 1e6, 2),
                                "ours_gcups_same_sample": round(ps * ps / rq.stats["ms_forward"] / 1e6, 1),
                                "vs_plain_full_step": round((n * m / (total / args.steps) / 1e9) /
                                                            (ps * ps / rp.stats["ms_forward"] / 1e6), 1)}

    if not args.no_extras and rank == 0:
        extras["small_pairs"] = bench_small_pairs(sw, ctx)
        extras["batch"] = bench_batch(sw, ctx)
        extras["serving"] = bench_serving(sw, ctx)

    if rank != 0:
        return
    value = _job_gcups(ws, n * m, args.steps, total)
    e2e = _job_gcups(ws, n * m, args.steps, e2e_total)
    fwd_s = statistics.mean(fwd_ms) / 1e3
    f_clk = (clk["sm_mhz"] or 2070) * 1e6
    import ctypes
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    achieved = statistics.mean(fwd_cells) * OPS_PER_CELL / fwd_s / 1e12
    peak = sms * INT_LANES_PER_CLK * f_clk / 1e12
    line = {
        "metric": "GCUPS", "value": round(value, 2), "unit": "GCUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total / args.steps * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
        "config": _config(n, m, ws),
        "result": {"score": r.score, "a": [r.a_begin, r.a_end], "b": [r.b_begin, r.b_end],
                   "cigar_len": len(r.cigar or "")},
        "phases_ms": {"forward": round(r.stats["ms_forward"], 1), "start": round(r.stats["ms_start"], 1),
                      "reconstruct": round(r.stats["ms_align"], 1), "levels": r.stats["levels"]},
        "roofline": {"bound": "alu", "kernel": "fwd16_kernel (forward score pass, int16x2 offset lanes, pruned)",
                     "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "Tops/s",
                     "frac": round(achieved / peak, 4), "traffic": FWD_TRAFFIC_BYTES,
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                     "cells_per_launch": int(statistics.mean(fwd_cells)), "ops_per_cell": OPS_PER_CELL,
                     "peak_basis": f"{sms} SMs x {INT_LANES_PER_CLK} int lane-ops/clk x {f_clk / 1e6:.0f} MHz (sampled)"},
        "e2e": {"value": round(e2e, 2), "unit": "GCUPS", "h2d_bytes_per_step": n + m,
                "d2h_bytes_per_step": len(re.cigar or "") + 96},
        "gpu_launches": launches,
        "clocks": clk,
        "extras": extras,
    }
    if ws == 1:
        line["cpu_baseline"] = cpu_baseline(a, b)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
