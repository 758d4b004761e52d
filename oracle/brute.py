"""Exhaustive enumeration of local alignments for tiny pairs (test pin).

Independent of ``sw_oracle.c``: no dynamic programming at all.  Every local
alignment of every pair of substrings is listed as an op string, scored with
the affine model, and the answers are selected by their definitions:

* S        = max(0, best score over all alignments);
* end      = smallest (a_end, b_end) among alignments scoring S;
* start    = largest (a_begin, b_begin) among those that end at `end`;
* path     = among alignments from start to end scoring S, the one whose
             backward sequence of choices is greatest under the preference
             "diagonal > vertical (I) > horizontal (D)" at a full cell and
             "open > extend" inside a gap -- the greedy traceback rule.

A gap run of k identical gap ops costs go + ge*(k-1) when go > ge (two
adjacent openings would cost more and are never optimal); when go == ge every
gap op is its own opening, which costs the same and is what "open > extend"
selects.  Practical up to about 5 x 5.
"""
from __future__ import annotations


def _score(ops, a, b, i0, j0, sub, go, ge):
    s, i, j, prev = 0, i0, j0, "M"
    for o in ops:
        if o == "M":
            s += sub[a[i]][b[j]]
            i += 1
            j += 1
        elif o == "I":
            s -= ge if (prev == "I" and go > ge) else go
            i += 1
        else:
            s -= ge if (prev == "D" and go > ge) else go
            j += 1
        prev = o
    return s


def _all_paths(n, m, i0, j0):
    """Every op string starting at (i0, j0) that stays inside the n x m grid."""
    out = []

    def rec(i, j, ops):
        out.append((i, j, "".join(ops)))
        if i < n and j < m:
            ops.append("M"); rec(i + 1, j + 1, ops); ops.pop()
        if i < n:
            ops.append("I"); rec(i + 1, j, ops); ops.pop()
        if j < m:
            ops.append("D"); rec(i, j + 1, ops); ops.pop()

    rec(i0, j0, [])
    return out


def _choice_ranks(ops, go, ge):
    """Backward sequence of greedy choice ranks for a path ending in state H."""
    ranks = []
    k = len(ops) - 1
    while k >= 0:
        o = ops[k]
        if o == "M":
            ranks.append(2)
            k -= 1
            continue
        ranks.append(1 if o == "I" else 0)        # H -> F (vertical) or H -> E
        run = 1
        if go > ge:
            while k - run >= 0 and ops[k - run] == o:
                run += 1
        ranks.extend([0] * (run - 1))             # extensions
        ranks.append(1)                            # the opening
        k -= run
    return ranks


def brute_local(a, b, sub, go, ge):
    """(S, a_begin, a_end, b_begin, b_end, ops) by exhaustive enumeration."""
    n, m = len(a), len(b)
    recs = []
    for i0 in range(n + 1):
        for j0 in range(m + 1):
            for (i1, j1, ops) in _all_paths(n, m, i0, j0):
                if ops:
                    recs.append((_score(ops, a, b, i0, j0, sub, go, ge), i0, j0, i1, j1, ops))
    S = max([0] + [r[0] for r in recs])
    if S == 0:
        return 0, -1, -1, -1, -1, ""
    opt = [r for r in recs if r[0] == S]
    end = min((r[3], r[4]) for r in opt)
    at_end = [r for r in opt if (r[3], r[4]) == end]
    start = max((r[1], r[2]) for r in at_end)
    cands = [r[5] for r in at_end if (r[1], r[2]) == start]
    best = max(cands, key=lambda o: _choice_ranks(o, go, ge))
    return S, start[0], end[0], start[1], end[1], best


def brute_global(a, b, sub, go, ge):
    """(value, ops) of the canonical optimal global alignment from H(0,0) to H(n,m)."""
    n, m = len(a), len(b)
    best_v, cands = None, []
    for (i1, j1, ops) in _all_paths(n, m, 0, 0):
        if (i1, j1) != (n, m):
            continue
        v = _score(ops, a, b, 0, 0, sub, go, ge)
        if best_v is None or v > best_v:
            best_v, cands = v, [ops]
        elif v == best_v:
            cands.append(ops)
    best = max(cands, key=lambda o: _choice_ranks(o, go, ge))
    return best_v, best
