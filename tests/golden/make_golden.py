"""Write the stored expected values under tests/golden/ (oracle only).

Every number written here comes from the CPU oracle (oracle/) run on inputs
from the seeded generator (gen/synth.py); nothing comes from the CUDA path.
The paper prints no worked example, score or alignment, so no value here is
the paper's own.

    python tests/golden/make_golden.py [pair_1k pair_100k batch_4096]

pair_1k     1,000 x ~1,000 pair: score, start/end, CIGAR
pair_100k   100,000 x ~100,000 pair: score, start/end, CIGAR length + sha256
batch_4096  4,096 pairs: score and end point per pair (score-only requests)
"""
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from gen import synth  # noqa: E402


def _write(name, obj):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(obj, f, indent=1)
        f.write("\n")


def pair(name, a, b, keep_cigar):
    t = time.time()
    r = oracle.align(a, b)
    rec = {"workload": name, "n": len(a), "m": len(b), "score": r.score,
           "a_begin": r.a_begin, "a_end": r.a_end, "b_begin": r.b_begin, "b_end": r.b_end,
           "cigar_len": len(r.cigar),
           "cigar_sha256": hashlib.sha256(r.cigar.encode()).hexdigest(),
           "scheme": {"match": 1, "mismatch": -3, "gap_open": 5, "gap_extend": 2},
           "source": "oracle/ (orc_local_score, orc_reverse_start, orc_global_trace)"}
    if keep_cigar:
        rec["cigar"] = r.cigar
    _write(f"{name}.json", rec)
    print(name, r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, f"{time.time() - t:.1f}s")


def _score_one(args):
    a, b = args
    return oracle.local_score(a, b)


def batch():
    t = time.time()
    pairs = synth.batch_pairs()
    ctx = mp.get_context("spawn")
    with ctx.Pool(os.cpu_count()) as pool:
        res = pool.map(_score_one, pairs, chunksize=8)
    _write("batch_4096.json", {
        "workload": "batch_4096", "count": len(pairs),
        "scheme": {"match": 1, "mismatch": -3, "gap_open": 5, "gap_extend": 2},
        "source": "oracle/ (orc_local_score)",
        "score_end": [[s, i, j] for (s, i, j) in res]})
    print("batch_4096", len(res), f"{time.time() - t:.1f}s")


if __name__ == "__main__":
    which = sys.argv[1:] or ["pair_1k", "pair_100k", "batch_4096"]
    oracle.build()
    if "pair_1k" in which:
        pair("pair_1k", *synth.pair_1k(), keep_cigar=True)
    if "pair_100k" in which:
        pair("pair_100k", *synth.pair_100k(), keep_cigar=False)
    if "batch_4096" in which:
        batch()
