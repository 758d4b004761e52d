"""Seeded synthetic DNA workloads for the affine-gap Smith-Waterman path.

This module only draws inputs. It does no alignment arithmetic; the oracle and
the CUDA path both take their inputs from here and from nowhere else.

Determinism across machines (x86_64 here, aarch64 on the GPU hosts) matters
because stored expected values are computed from these inputs on one machine
and compared on another.  Every random draw is therefore a counter-based
splitmix64 hash of (seed, stream, index) evaluated in wrapping uint64
arithmetic; probabilities are integer thresholds; the two places that need a
transcendental (log-uniform lengths and exponential inter-arrival times) use
`_exp`/`_ln` below, written with IEEE-754 +, -, *, / only, which are correctly
rounded everywhere.

Codes: 0=A, 1=C, 2=G, 3=T (uint8).  `decode`/`encode` convert to/from ASCII.

Workload recipes (the paper's Table 1 pairs are real chromosomes that are not
available; these stand in for them, bracketing their 0.16-59 Mb sizes):

* ``pair_1k``      A = 1,000 uniform bases; B = 800-base window of A at a random
                   offset, mutated, flanked by 100 random bases on each side.
* ``pair_100k``    A = 100,000 uniform bases with 5 % of positions overwritten by
                   tandem repeats (unit 2-50, copies 2-20); B = A mutated.
* ``pair_5m``      A = 5,000,000 bases at GC 41 % with the same repeats; B = A
                   mutated, then a 20 kbp inversion (reverse complement) and a
                   50 kbp deletion at random non-overlapping sites.
* ``batch_4096``   4,096 pairs, lengths log-uniform in [100, 20,000] per side;
                   even-indexed pairs homologous (B = mutated window of A of
                   length min(la, lb), padded with random bases to lb), odd
                   pairs unrelated.
* ``serve_stream`` Poisson arrivals; one length L log-uniform in [1e3, 1e6] per
                   request, B = A mutated; 70 % score-only, 30 % alignment.

Mutation model (per source base, in order): with probability 10 % substitute
one of the other three bases; 1 % start a deletion; 1 % insert random bases
before the base.  Indel lengths are geometric with success probability 1/3
(mean 3), capped at 60.  A deletion swallows the following bases and their own
draws.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)

ALPHABET = "ACGT"
_ENC = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(ALPHABET):
    _ENC[ord(_c)] = _i
    _ENC[ord(_c.lower())] = _i
_ENC[ord("N")] = 4
_ENC[ord("n")] = 4


def encode(s: str | bytes) -> np.ndarray:
    """ASCII bases -> codes (A0 C1 G2 T3 N4); other bytes raise ValueError."""
    if isinstance(s, str):
        s = s.encode()
    out = _ENC[np.frombuffer(s, dtype=np.uint8)]
    if (out == 255).any():
        raise ValueError("non-DNA character in sequence")
    return out


def decode(codes: np.ndarray) -> str:
    return bytes(np.frombuffer(b"ACGTN", dtype=np.uint8)[np.asarray(codes)]).decode()


def _mix(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea & Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        x = x ^ (x >> np.uint64(30))
        x = x * np.uint64(0xBF58476D1CE4E5B9)
        x = x ^ (x >> np.uint64(27))
        x = x * np.uint64(0x94D049BB133111EB)
        x = x ^ (x >> np.uint64(31))
    return x


class Rng:
    """Counter-based stream: draw k of stream s is mix(seed*G + s*K + k)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self._next_stream = 1

    def stream(self) -> "Stream":
        s = self._next_stream
        self._next_stream += 1
        return Stream(self.seed, s)


class Stream:
    def __init__(self, seed: np.uint64, stream: int):
        with np.errstate(over="ignore"):
            self.base = seed * _GOLD + np.uint64(stream) * _STREAM
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.pos, self.pos + n, dtype=np.uint64)
        self.pos += n
        with np.errstate(over="ignore"):
            return _mix(idx + self.base)

    def below(self, n: int, k: int) -> np.ndarray:
        """n draws uniform in [0, k) (k << 2**32: modulo bias < 2**-32)."""
        return (self.u64(n) >> np.uint64(32)) % np.uint64(k)

    def unit(self, n: int) -> np.ndarray:
        """n float64 draws uniform in [0, 1) with 53 random bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def int(self, lo: int, hi: int) -> int:
        """One integer uniform in [lo, hi] inclusive."""
        return lo + int(self.below(1, hi - lo + 1)[0])


def _exp(x: float) -> float:
    """exp(x) with basic IEEE operations only (range reduction by ln 2)."""
    ln2 = 0.6931471805599453
    k = int(x / ln2 + (0.5 if x >= 0 else -0.5))
    r = x - k * ln2
    term, total = 1.0, 1.0
    for i in range(1, 25):
        term = term * r / i
        total += term
    return total * (2.0 ** k)


def _ln(x: float) -> float:
    """ln(x) for x > 0 with basic IEEE operations only (atanh series)."""
    if x <= 0:
        raise ValueError("ln of non-positive")
    k = 0
    while x > 2.0:
        x /= 2.0
        k += 1
    while x < 1.0:
        x *= 2.0
        k -= 1
    y = (x - 1.0) / (x + 1.0)
    y2, term, total = y * y, y, 0.0
    for i in range(60):
        total += term / (2 * i + 1)
        term *= y2
    return 2.0 * total + k * 0.6931471805599453


def log_uniform_int(st: Stream, lo: int, hi: int, n: int) -> np.ndarray:
    """n integers log-uniform in [lo, hi]: floor(lo * (hi/lo)**u), clamped."""
    u = st.unit(n)
    lr = _ln(hi / lo)
    out = np.empty(n, dtype=np.int64)
    for t in range(n):
        out[t] = min(hi, max(lo, int(lo * _exp(float(u[t]) * lr))))
    return out


def random_bases(st: Stream, n: int, gc_permille: int | None = None) -> np.ndarray:
    """n bases; uniform, or with P(G)=P(C)=gc/2 when gc_permille is given."""
    if gc_permille is None:
        return st.below(n, 4).astype(np.uint8)
    d = st.below(n, 1000).astype(np.int64)
    at = (1000 - gc_permille) // 2
    gc = gc_permille // 2
    out = np.full(n, 3, dtype=np.uint8)              # T
    out[d < at + 2 * gc] = 2                           # G
    out[d < at + gc] = 1                               # C
    out[d < at] = 0                                    # A
    return out


def _geometric(st: Stream, n: int, cap: int = 60) -> np.ndarray:
    """n lengths >= 1, geometric with success probability 1/3, capped."""
    if n == 0:
        return np.zeros(0, dtype=np.int64)
    trials = st.below(n * cap, 3).reshape(n, cap)
    succ = trials == 0
    first = np.where(succ.any(axis=1), succ.argmax(axis=1), cap - 1)
    return first.astype(np.int64) + 1


def add_tandem_repeats(st: Stream, seq: np.ndarray, frac_permille: int = 50,
                       gc_permille: int | None = None) -> np.ndarray:
    """Overwrite ~frac of positions with tandem repeats (unit 2-50, copies 2-20)."""
    seq = seq.copy()
    L = len(seq)
    target = L * frac_permille // 1000
    written = 0
    while written < target and L > 4:
        unit = st.int(2, 50)
        copies = st.int(2, 20)
        pos = st.int(0, L - 1)
        motif = random_bases(st, unit, gc_permille)
        rep = np.tile(motif, copies)[: L - pos]
        seq[pos: pos + len(rep)] = rep
        written += len(rep)
    return seq


def mutate(st: Stream, src: np.ndarray, sub_permille: int = 100,
           del_permille: int = 10, ins_permille: int = 10,
           gc_permille: int | None = None) -> np.ndarray:
    """Apply the per-base substitution / deletion / insertion model to src."""
    n = len(src)
    if n == 0:
        return src.copy()
    ev = st.below(n, 1000).astype(np.int64)
    alt = st.below(n, 3).astype(np.uint8)
    is_sub = ev < sub_permille
    is_del = (ev >= sub_permille) & (ev < sub_permille + del_permille)
    is_ins = (ev >= sub_permille + del_permille) & (ev < sub_permille + del_permille + ins_permille)
    out = src.copy()
    out[is_sub] = (src[is_sub] + 1 + alt[is_sub]) % 4
    keep = np.ones(n, dtype=bool)
    del_pos = np.nonzero(is_del)[0]
    del_len = _geometric(st, len(del_pos))
    covered_until = -1
    for p, k in zip(del_pos.tolist(), del_len.tolist()):
        if p <= covered_until:
            continue  # swallowed by an earlier deletion
        keep[p: p + k] = False
        covered_until = p + k - 1
    ins_pos = np.nonzero(is_ins & keep)[0]
    ins_len = _geometric(st, len(ins_pos))
    ins_total = int(ins_len.sum())
    ins_bases = random_bases(st, ins_total, gc_permille)
    pieces = []
    prev = 0
    off = 0
    for p, k in zip(ins_pos.tolist(), ins_len.tolist()):
        pieces.append(out[prev:p][keep[prev:p]])
        pieces.append(ins_bases[off: off + k])
        off += k
        prev = p
    pieces.append(out[prev:][keep[prev:]])
    return np.concatenate(pieces).astype(np.uint8)


def revcomp(seq: np.ndarray) -> np.ndarray:
    return (3 - seq[::-1]).astype(np.uint8)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def pair_1k(seed: int = 1):
    """1,000-base A; B = mutated 800-base window of A flanked by 100 random bases."""
    r = Rng(seed)
    st = r.stream()
    a = random_bases(st, 1000)
    off = st.int(0, 200)
    core = mutate(r.stream(), a[off: off + 800])
    fl = r.stream()
    b = np.concatenate([random_bases(fl, 100), core, random_bases(fl, 100)]).astype(np.uint8)
    return a, b


def pair_homologous(length: int, seed: int, gc_permille: int | None = None,
                    repeats: bool = True):
    """A of `length` (tandem repeats on 5 %); B = A mutated."""
    r = Rng(seed)
    a = random_bases(r.stream(), length, gc_permille)
    if repeats:
        a = add_tandem_repeats(r.stream(), a, 50, gc_permille)
    b = mutate(r.stream(), a, gc_permille=gc_permille)
    return a, b


def pair_100k(seed: int = 2):
    return pair_homologous(100_000, seed)


def pair_5m(seed: int = 3, length: int = 5_000_000, inversion: int = 20_000,
            deletion: int = 50_000):
    """Chromosome-scale pair: GC 41 %, repeats, mutation, inversion, deletion."""
    a, b = pair_homologous(length, seed, gc_permille=410)
    st = Rng(seed ^ 0x5F5F).stream()
    L = len(b)
    if L > 4 * (inversion + deletion):
        # two non-overlapping sites: inversion in the first half, deletion in the second
        s_inv = st.int(0, L // 2 - inversion - 1)
        s_del = st.int(L // 2, L - deletion - 1)
        b = b.copy()
        b[s_inv: s_inv + inversion] = revcomp(b[s_inv: s_inv + inversion])
        b = np.concatenate([b[:s_del], b[s_del + deletion:]]).astype(np.uint8)
    return a, b


def batch_pairs(count: int = 4096, seed: int = 4, lo: int = 100, hi: int = 20_000):
    """`count` pairs, lengths log-uniform per side; even homologous, odd unrelated."""
    r = Rng(seed)
    lst = r.stream()
    la = log_uniform_int(lst, lo, hi, count)
    lb = log_uniform_int(lst, lo, hi, count)
    pairs = []
    for t in range(count):
        st = r.stream()
        a = random_bases(st, int(la[t]))
        if t % 2 == 0:
            w = int(min(la[t], lb[t]))
            off = st.int(0, int(la[t]) - w)
            core = mutate(st, a[off: off + w])[: int(lb[t])]
            pad = int(lb[t]) - len(core)
            left = st.int(0, pad) if pad > 0 else 0
            b = np.concatenate([random_bases(st, left), core,
                                random_bases(st, pad - left)]).astype(np.uint8)
        else:
            b = random_bases(st, int(lb[t]))
        pairs.append((a, b))
    return pairs


def serve_stream(count: int, rate_per_s: float, seed: int = 5, lo: int = 1_000,
                 hi: int = 1_000_000):
    """`count` requests: (arrival_s, a, b, align_flag) with Poisson arrivals."""
    r = Rng(seed)
    st = r.stream()
    u = st.unit(count)
    kinds = st.below(count, 100)
    lens = log_uniform_int(st, lo, hi, count)
    t = 0.0
    out = []
    for k in range(count):
        t += -_ln(1.0 - float(u[k])) / rate_per_s
        a, b = pair_homologous(int(lens[k]), seed * 1_000_003 + k, repeats=False)
        out.append((t, a, b, bool(kinds[k] >= 70)))
    return out


def random_pair(n: int, m: int, seed: int, alphabet: int = 4):
    """Independent uniform sequences (used for small randomized parity cases)."""
    st = Rng(seed).stream()
    a = st.below(n, alphabet).astype(np.uint8)
    b = st.below(m, alphabet).astype(np.uint8)
    return a, b


def related_pair(n: int, seed: int, sub_permille: int = 100):
    """A uniform of length n; B = A mutated (small homologous parity cases)."""
    r = Rng(seed)
    a = random_bases(r.stream(), n)
    b = mutate(r.stream(), a, sub_permille=sub_permille)
    return a, b
