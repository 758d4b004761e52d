"""Pins for the CPU oracle against facts that do not come from the oracle itself.

* exhaustive enumeration of every local / global alignment on tiny pairs
  (oracle/brute.py, no dynamic programming);
* closed forms: identical sequences, homopolymers, all-mismatch, one
  substitution, one inserted run;
* symmetry and reversal invariants;
* the rescoring invariant (the emitted alignment scores exactly S and consumes
  exactly [begin, end));
* the sub-path property of the greedy traceback (its segment between two of
  its nodes is the traceback of that sub-problem), which pins the E/F source
  and sink handling;
* the streaming verifier accepts exactly one of all optimal paths.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import brute
from gen import synth

SCHEMES = [
    oracle.Scheme(1, -3, 5, 2),
    oracle.Scheme(2, -1, 2, 1),
    oracle.Scheme(1, -1, 1, 1),     # go == ge: linear gaps
    oracle.Scheme(3, -2, 4, 1),
]


def _sub(sch):
    return sch.table().tolist()


def _check_vs_brute(a, b, sch):
    S, ab, ae, bb, be, ops = brute.brute_local(list(a), list(b), _sub(sch), sch.gap_open, sch.gap_extend)
    got = oracle.align(np.array(a, dtype=np.uint8), np.array(b, dtype=np.uint8), sch)
    assert (got.score, got.a_begin, got.a_end, got.b_begin, got.b_end) == (S, ab, ae, bb, be), (a, b, sch)
    if S:
        assert oracle.cigar_to_ops(got.cigar) == ops, (a, b, sch, got.cigar, ops)


@pytest.mark.parametrize("sch", SCHEMES)
def test_exhaustive_binary_pairs(sch):
    # every pair over a 2-letter alphabet up to length 3: many ties
    for n in range(0, 4):
        for m in range(0, 4):
            for a in itertools.product([0, 1], repeat=n):
                for b in itertools.product([0, 1], repeat=m):
                    _check_vs_brute(a, b, sch)


@pytest.mark.parametrize("sch", SCHEMES)
def test_random_tiny_vs_brute(sch):
    st = synth.Rng(11).stream()
    for t in range(40):
        n = int(st.below(1, 5)[0]) + 1
        m = int(st.below(1, 5)[0]) + 1
        alph = 2 if t % 2 else 4
        a = st.below(n, alph).astype(np.uint8)
        b = st.below(m, alph).astype(np.uint8)
        _check_vs_brute(a, b, sch)


@pytest.mark.parametrize("sch", SCHEMES[:2])
def test_global_vs_brute(sch):
    st = synth.Rng(12).stream()
    for t in range(60):
        n = int(st.below(1, 5)[0])
        m = int(st.below(1, 5)[0])
        a = st.below(n, 2).astype(np.uint8)
        b = st.below(m, 2).astype(np.uint8)
        v, ops = brute.brute_global(list(a), list(b), _sub(sch), sch.gap_open, sch.gap_extend)
        v2, ops2 = oracle.global_trace(a, b, sch)
        assert (v2, ops2) == (v, ops), (a, b)


def test_closed_form_identical():
    for L in (1, 2, 7, 100, 513):
        a = synth.random_pair(L, 1, seed=L)[0]
        r = oracle.align(a, a)
        assert (r.score, r.a_begin, r.a_end, r.b_begin, r.b_end, r.cigar) == (L, 0, L, 0, L, f"{L}=")


def test_closed_form_homopolymer():
    for n, m in [(5, 9), (9, 5), (1, 30), (64, 64)]:
        a = np.zeros(n, np.uint8)
        b = np.zeros(m, np.uint8)
        S, ei, ej = oracle.local_score(a, b)
        k = min(n, m)
        assert (S, ei, ej) == (k, k, k)


def test_closed_form_all_mismatch():
    # disjoint alphabets via the matrix: every substitution negative
    mat = tuple([-1] * 16)
    sch = oracle.Scheme(alphabet=4, matrix=mat)
    a, b = synth.random_pair(50, 60, seed=3)
    assert oracle.local_score(a, b, sch)[0] == 0
    r = oracle.align(a, b, sch)
    assert (r.score, r.a_begin, r.cigar) == (0, -1, "")


def test_closed_form_one_substitution():
    # A = B except one mismatch at p: S = max(L - 4, p, L - p - 1)
    for L, p in [(20, 0), (20, 3), (20, 10), (20, 19), (9, 4), (5, 2)]:
        a = synth.random_pair(L, 1, seed=100 + L)[0]
        b = a.copy()
        b[p] = (b[p] + 1) % 4
        S = oracle.local_score(a, b)[0]
        assert S == max(L - 4, p, L - p - 1), (L, p, S)


def test_closed_form_inserted_run():
    # B = X G Y, A = X Y, G over code 4 which mismatches everything (matrix):
    # S = max(L - (go + ge*(k-1)), |X|, |Y|) with go=5, ge=2 -> 3 + 2k for the gap
    mat = [[1 if (x == y and x < 4) else -3 for y in range(5)] for x in range(5)]
    sch = oracle.Scheme(alphabet=5, matrix=tuple(v for row in mat for v in row))
    for nx, ny, k in [(10, 10, 1), (10, 10, 3), (4, 30, 2), (25, 3, 5), (8, 8, 12)]:
        x = synth.random_pair(nx, 1, seed=nx * 7 + k)[0]
        y = synth.random_pair(ny, 1, seed=ny * 11 + k)[0]
        a = np.concatenate([x, y]).astype(np.uint8)
        b = np.concatenate([x, np.full(k, 4, np.uint8), y]).astype(np.uint8)
        S = oracle.local_score(a, b, sch)[0]
        assert S == max(nx + ny - (5 + 2 * (k - 1)), nx, ny), (nx, ny, k, S)


def test_symmetry_and_reversal():
    for seed in range(8):
        a, b = synth.related_pair(300, seed=seed)
        S = oracle.local_score(a, b)[0]
        assert oracle.local_score(b, a)[0] == S
        assert oracle.local_score(a[::-1].copy(), b[::-1].copy())[0] == S


def test_rescore_invariant_and_verifier():
    for seed in range(6):
        a, b = synth.related_pair(400, seed=20 + seed)
        r = oracle.align(a, b)
        ops = oracle.cigar_to_ops(r.cigar)
        s, ua, ub = oracle.rescore(a[r.a_begin:r.a_end], b[r.b_begin:r.b_end], ops)
        assert (s, ua, ub) == (r.score, r.a_end - r.a_begin, r.b_end - r.b_begin)
        assert oracle.verify_path(a[r.a_begin:r.a_end], b[r.b_begin:r.b_end], ops) == 0
        # the end point carries S and nothing exceeds it in the reverse pass
        bi, bj, mx = oracle.reverse_start(a, b, r.a_end, r.b_end, r.score, scan_all=True)
        assert (bi, bj) == (r.a_begin, r.b_begin) and mx == r.score


def test_pair_1k_alignment_is_consistent():
    a, b = synth.pair_1k()
    r = oracle.align(a, b)
    assert r.score > 300          # ~800 homologous bases at 10 % substitution
    ops = oracle.cigar_to_ops(r.cigar)
    assert oracle.rescore(a[r.a_begin:r.a_end], b[r.b_begin:r.b_end], ops)[0] == r.score
    # alignment neither begins nor ends with a gap (go > 0)
    assert ops[0] == "M" and ops[-1] == "M"


@pytest.mark.parametrize("sch", [oracle.Scheme(1, -1, 1, 1), oracle.Scheme(2, -1, 2, 1),
                                 oracle.Scheme(1, -3, 5, 2), oracle.Scheme(3, -1, 3, 1)])
def test_verifier_accepts_exactly_one_optimal_path(sch):
    # every binary pair of these shapes: all complete paths are enumerated and
    # the verifier must accept the brute-force canonical one and nothing else
    # (5 x 2 and 2 x 5 contain open/extend ties inside gap runs)
    for n, m in [(3, 4), (5, 2), (2, 5)]:
        paths = [p[2] for p in brute._all_paths(n, m, 0, 0) if p[:2] == (n, m)]
        for a in itertools.product([0, 1], repeat=n):
            for b in itertools.product([0, 1], repeat=m):
                a_, b_ = np.array(a, np.uint8), np.array(b, np.uint8)
                v, canon = brute.brute_global(list(a), list(b), _sub(sch), sch.gap_open, sch.gap_extend)
                accepted = [ops for ops in paths if oracle.verify_path(a_, b_, ops, sch) == 0]
                assert accepted == [canon], (a, b, sch, accepted, canon)


def _nodes_along(ops, go, ge):
    """(i, j, state, index into ops) for nodes in the middle of the path."""
    out, i, j, prev = [], 0, 0, "M"
    for k, o in enumerate(ops):
        if o == "M":
            i += 1; j += 1; st = oracle.H
        elif o == "I":
            i += 1; st = oracle.F
        else:
            j += 1; st = oracle.E
        out.append((i, j, st, k + 1))
        prev = o
    return out


@pytest.mark.parametrize("sch", [oracle.DNA, oracle.Scheme(1, -1, 1, 1), oracle.Scheme(2, -1, 2, 1)])
def test_subpath_property_with_gap_states(sch):
    """Segment of the canonical path between two of its nodes == traceback of that sub-problem."""
    checked = 0
    for seed in range(10):
        a, b = synth.related_pair(220, seed=50 + seed, sub_permille=150)
        # force long gaps so that E/F nodes appear
        b = np.concatenate([b[:60], b[75:150], synth.random_pair(9, 1, seed=seed)[0], b[150:]]).astype(np.uint8)
        v, ops = oracle.global_trace(a, b, sch)
        nodes = _nodes_along(ops, sch.gap_open, sch.gap_extend)
        gap_nodes = [x for x in nodes if x[2] != oracle.H]
        picks = gap_nodes[:: max(1, len(gap_nodes) // 4)] + nodes[:: max(1, len(nodes) // 5)]
        for (i0, j0, s0, k0) in picks:
            for (i1, j1, s1, k1) in picks:
                if k1 <= k0:
                    continue
                # a node inside a gap run is in the gap state; a node that ends
                # a run and is followed by another op also exists in state H
                seg = ops[k0:k1]
                val, sub_ops = oracle.global_trace(a[i0:i1], b[j0:j1], sch, src=s0, snk=s1)
                assert sub_ops == seg, (seed, i0, j0, s0, i1, j1, s1)
                assert oracle.rescore(a[i0:i1], b[j0:j1], seg, sch, src=s0)[0] == val
                assert oracle.verify_path(a[i0:i1], b[j0:j1], seg, sch, src=s0, snk=s1) == 0
                checked += 1
    assert checked > 50


def test_verifier_rejects_planted_mistakes():
    a, b = synth.related_pair(300, seed=77)
    r = oracle.align(a, b)
    asub, bsub = a[r.a_begin:r.a_end], b[r.b_begin:r.b_end]
    ops = oracle.cigar_to_ops(r.cigar)
    # swap an adjacent "MI" -> "IM" somewhere, or flip a diagonal into two gaps
    k = ops.find("MI")
    if k >= 0:
        bad = ops[:k] + "IM" + ops[k + 2:]
        assert oracle.verify_path(asub, bsub, bad) != 0
    k = ops.find("M", 5)
    bad = ops[:k] + "ID" + ops[k + 1:]
    assert oracle.verify_path(asub, bsub, bad) != 0
    assert oracle.verify_path(asub, bsub, ops[:-1]) != 0
