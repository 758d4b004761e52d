"""The seeded input generator (gen/synth.py) follows its stated recipe.

Every parity case and benchmark input comes from this module, so its rates are
checked here against the recipe: substitutions 10 %, deletion and insertion
starts 1 % each with geometric lengths of mean 3, GC 41 % for the
chromosome-scale pair, log-uniform lengths, Poisson arrivals with 30 %
alignment requests.  Tolerances are several binomial standard deviations.
"""
import math

import numpy as np
import pytest

from gen import synth


def test_deterministic_and_seeded():
    a1, b1 = synth.pair_1k()
    a2, b2 = synth.pair_1k()
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    a3, _ = synth.pair_1k(seed=11)
    assert not np.array_equal(a1, a3)
    st1, st2 = synth.Rng(7).stream(), synth.Rng(7).stream()
    assert np.array_equal(st1.u64(1000), st2.u64(1000))


def test_exp_and_ln_match_the_math_library():
    for x in np.linspace(-40.0, 40.0, 801):
        assert synth._exp(float(x)) == pytest.approx(math.exp(x), rel=1e-13)
    for x in np.geomspace(1e-6, 1e9, 801):
        assert synth._ln(float(x)) == pytest.approx(math.log(x), rel=1e-13, abs=1e-15)


def test_encode_decode_and_revcomp():
    s = "ACGTNacgtn"
    assert synth.decode(synth.encode(s)) == s.upper()
    with pytest.raises(ValueError):
        synth.encode("ACGU")
    x = synth.random_bases(synth.Rng(3).stream(), 1000)
    assert np.array_equal(synth.revcomp(synth.revcomp(x)), x)
    assert synth.decode(synth.revcomp(synth.encode("AACGT"))) == "ACGTT"


def test_substitution_rate():
    st = synth.Rng(21).stream()
    src = synth.random_bases(st, 1_000_000)
    out = synth.mutate(st, src, sub_permille=100, del_permille=0, ins_permille=0)
    assert len(out) == len(src)
    diff = out != src
    assert abs(diff.mean() - 0.100) < 0.002
    # the substituted base is one of the other three, each equally likely
    shift = ((out[diff].astype(int) - src[diff].astype(int)) % 4)
    counts = np.bincount(shift, minlength=4)
    assert counts[0] == 0 and all(abs(c / diff.sum() - 1 / 3) < 0.01 for c in counts[1:])


def test_insertion_and_deletion_lengths():
    st = synth.Rng(22).stream()
    L = 1_000_000
    src = synth.random_bases(st, L)
    ins = synth.mutate(st, src, sub_permille=0, del_permille=0, ins_permille=10)
    # 1 % of bases start an insertion of mean length 3
    assert abs((len(ins) - L) / L - 0.030) < 0.002
    dele = synth.mutate(st, src, sub_permille=0, del_permille=10, ins_permille=0)
    # a deletion of mean length 3 starts at 1 % of the bases not already deleted:
    # deleted fraction 0.01 * 3 / (0.99 + 0.01 * 3)
    assert abs((L - len(dele)) / L - 0.03 / 1.02) < 0.002
    g = synth._geometric(st, 200_000)
    assert g.min() == 1 and g.max() <= 60 and abs(g.mean() - 3.0) < 0.05


def test_gc_content_and_chromosome_pair():
    st = synth.Rng(23).stream()
    x = synth.random_bases(st, 1_000_000, gc_permille=410)
    gc = np.isin(x, [1, 2]).mean()
    assert abs(gc - 0.41) < 0.003
    assert abs((x == 1).mean() - (x == 2).mean()) < 0.003
    a, b = synth.pair_5m()
    assert len(a) == 5_000_000
    # B = A mutated (insertions and deletions nearly cancel) minus the 50 kbp deletion
    assert abs(len(b) - (len(a) - 50_000)) < 10_000
    assert abs(np.isin(a, [1, 2]).mean() - 0.41) < 0.003


def test_batch_lengths_log_uniform():
    st = synth.Rng(4).stream()
    L = synth.log_uniform_int(st, 100, 20_000, 20_000)
    assert L.min() >= 100 and L.max() <= 20_000
    # ln L is uniform on [ln 100, ln 20000]: mean at the midpoint, median at sqrt(100 * 20000)
    assert abs(np.log(L).mean() - 0.5 * (math.log(100) + math.log(20_000))) < 0.05
    assert abs((L < math.sqrt(100 * 20_000)).mean() - 0.5) < 0.02


def test_serve_stream_arrivals_and_mix():
    rate = 50.0
    reqs = synth.serve_stream(600, rate, seed=9, lo=60, hi=80)
    t = np.array([r[0] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() * rate - 1.0) < 0.15            # exponential gaps of mean 1/rate
    assert abs(np.std(gaps) * rate - 1.0) < 0.2
    align = np.mean([r[3] for r in reqs])
    assert abs(align - 0.30) < 0.06
    assert all(60 <= len(r[1]) <= 80 for r in reqs)
