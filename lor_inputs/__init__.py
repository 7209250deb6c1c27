"""Seeded synthetic DNA inputs shared by the tests, the benchmark and the smoke
check.

This module only draws random sequences; it holds none of the method's
arithmetic (no coding, sorting or comparison).  Sequences are returned as
ASCII ``uint8`` numpy arrays over ``ACGT``.  The paper evaluates on three NCBI
noncoding accessions that are not available here; these generators stand in
for them with the shapes the workloads name:

* ``pair_uniform``     -- two iid uniform sequences with one planted exact
  common substring (the 2 x 100,000 and 2 x 134,217,728 base instances);
* ``pair_noncoding``   -- two sequences shaped like noncoding DNA: 40 % GC
  background, ~10 % interspersed copies of five 300-bp consensus repeats at
  10-20 % point mutation, ~3 % microsatellites (period 1-6, 10-60 copies),
  and one shared 10 kb region with 1 % mutations around an exact 2 kb core;
* ``pair_batch``       -- many pairs of uneven, log-uniform length;
* ``multi_query``      -- one reference and many query sequences (reads of
  the reference with substitutions, and background with a planted piece);
* ``pair_int64``       -- two uniform sequences whose concatenation passes
  2^31 symbols (the 64-bit index path), and ``random_queries64``;
* ``random_queries``   -- uniform (p, q) suffix pairs for LCP queries;
* ``poisson_arrivals`` -- request arrival times of a Poisson process, and
  ``request_stream``   -- which pool pair each arrival asks for and its
  follow-up LCP queries (the served workload);
* ``fuzz_pair``        -- small random/degenerate cases for parity tests.

Seeds: workload c (1-based) uses seed 140434480 + c unless given another.
"""
from __future__ import annotations

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
SEED_BASE = 140434480

SIZE_TINY = 100_000
SIZE_NONCODING = 16_777_216
SIZE_LARGE = 134_217_728


def _rng(seed):
    return np.random.default_rng(seed)


def random_bases(rng, n, probs=None) -> np.ndarray:
    """n bases; iid uniform, or with probabilities for A, C, G, T."""
    if probs is None:
        idx = rng.integers(0, 4, size=n, dtype=np.uint8)
    else:
        idx = rng.choice(4, size=n, p=probs).astype(np.uint8)
    return ACGT[idx]


def mutate(rng, seq, rate) -> np.ndarray:
    """Copy of seq with independent point substitutions at ``rate``; a
    substituted base is drawn uniformly from the three other bases."""
    out = seq.copy()
    hit = np.flatnonzero(rng.random(seq.size) < rate)
    if hit.size:
        code = np.searchsorted(ACGT, out[hit])          # A,C,G,T -> 0..3
        shift = rng.integers(1, 4, size=hit.size)
        out[hit] = ACGT[(code + shift) % 4]
    return out


def _plant(rng, seq, piece):
    if piece.size == 0 or piece.size > seq.size:
        return -1
    off = int(rng.integers(0, seq.size - piece.size + 1))
    seq[off:off + piece.size] = piece
    return off


def pair_uniform(n_each=SIZE_TINY, plant_len=500, seed=SEED_BASE + 1):
    """Two iid uniform sequences of ``n_each`` bases; one exact substring of
    ``plant_len`` bases planted at a uniform offset in each.  Returns
    ([s1, s2], info)."""
    rng = _rng(seed)
    s1 = random_bases(rng, n_each)
    s2 = random_bases(rng, n_each)
    plant_len = min(plant_len, n_each)
    piece = random_bases(rng, plant_len)
    o1 = _plant(rng, s1, piece)
    o2 = _plant(rng, s2, piece)
    return [s1, s2], dict(plant_len=plant_len, plant_offsets=(o1, o2), seed=seed)


NONCODING_PROBS = (0.3, 0.2, 0.2, 0.3)


def noncoding_sequence(rng, n, consensi, shared=None, core=2000, shared_rate=0.01):
    """One noncoding-like sequence of n bases (see module docstring)."""
    s = random_bases(rng, n, NONCODING_PROBS)
    # interspersed repeats: ~10 % of the sequence, 10-20 % substitutions each
    if consensi:
        clen = len(consensi[0])
        copies = int(round(0.10 * n / clen)) if n >= clen else 0
        for _ in range(copies):
            cons = consensi[int(rng.integers(0, len(consensi)))]
            _plant(rng, s, mutate(rng, cons, float(rng.uniform(0.10, 0.20))))
    # microsatellites: ~3 % of the sequence, unit period 1-6, 10-60 copies
    target, covered = 0.03 * n, 0
    while covered < target:
        period = int(rng.integers(1, 7))
        unit = random_bases(rng, period)
        rep = np.tile(unit, int(rng.integers(10, 61)))
        if rep.size > n:
            break
        _plant(rng, s, rep)
        covered += rep.size
    # shared region, planted last: 1 % substitutions outside an exact core
    off = -1
    if shared is not None and shared.size <= n:
        copy = mutate(rng, shared, shared_rate)
        c0 = (shared.size - core) // 2
        if core > 0:
            copy[c0:c0 + core] = shared[c0:c0 + core]
        off = _plant(rng, s, copy)
    return s, off


def pair_noncoding(n_each=SIZE_NONCODING, seed=SEED_BASE + 2, shared_len=10_000, core=2000):
    """Two noncoding-like sequences sharing five consensus repeat families and
    one 10 kb region (exact 2 kb core).  Returns ([s1, s2], info)."""
    rng = _rng(seed)
    consensi = [random_bases(rng, 300) for _ in range(5)]
    shared_len = min(shared_len, n_each)
    core = min(core, shared_len)
    shared = random_bases(rng, shared_len)
    s1, o1 = noncoding_sequence(rng, n_each, consensi, shared, core)
    s2, o2 = noncoding_sequence(rng, n_each, consensi, shared, core)
    return [s1, s2], dict(shared_len=shared_len, core=core, shared_offsets=(o1, o2), seed=seed)


def pair_large(n_each=SIZE_LARGE, seed=SEED_BASE + 3, plant_len=500):
    """Two iid uniform sequences of 134,217,728 bases with one 500-base plant
    (the same generator as the 2 x 100,000 instance)."""
    return pair_uniform(n_each=n_each, plant_len=plant_len, seed=seed)


# Past the int32 index range: n = 2 * (2^30 + 2^15) + 2 = 2^31 + 2^16 + 2.
SIZE_INT64 = (1 << 30) + (1 << 15)


def pair_int64(n_each=SIZE_INT64, seed=SEED_BASE + 8, plant_len=500):
    """Two iid uniform sequences whose concatenation passes 2^31 symbols, with
    one 500-base plant at a uniform offset in the first and 600 bases before
    the end of the second, so that its text position there lies past 2^31."""
    rng = _rng(seed)
    s1 = random_bases(rng, n_each)
    s2 = random_bases(rng, n_each)
    piece = random_bases(rng, plant_len)
    o1 = _plant(rng, s1, piece)
    o2 = n_each - plant_len - 100
    s2[o2:o2 + plant_len] = piece
    return [s1, s2], dict(plant_len=plant_len, plant_offsets=(o1, o2), seed=seed)


def random_queries64(n, count=1_000_000, seed=SEED_BASE + 8):
    """``count`` (p, q) pairs uniform in [0, n)^2 (int64)."""
    rng = _rng(seed + 1000)
    return (rng.integers(0, n, size=count, dtype=np.int64), rng.integers(0, n, size=count, dtype=np.int64))


def random_queries(n, count=1_000_000, seed=SEED_BASE + 3):
    """``count`` (p, q) pairs uniform in [0, n)^2 (int32)."""
    rng = _rng(seed + 1000)
    p = rng.integers(0, n, size=count, dtype=np.int64).astype(np.int32)
    q = rng.integers(0, n, size=count, dtype=np.int64).astype(np.int32)
    return p, q


def pair_batch(npairs=4096, lo=1_000, hi=1_000_000, seed=SEED_BASE + 4):
    """``npairs`` pairs of noncoding-like sequences with per-sequence lengths
    log-uniform in [lo, hi] and one shared planted region per pair of length
    uniform in [50, 5000] (clamped to the shorter sequence)."""
    rng = _rng(seed)
    consensi = [random_bases(rng, 300) for _ in range(5)]
    pairs = []
    for _ in range(npairs):
        l1, l2 = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(2))
        plen = min(int(rng.integers(50, 5001)), l1, l2)
        shared = random_bases(rng, plen)
        s1, _ = noncoding_sequence(rng, l1, consensi, shared, core=plen)
        s2, _ = noncoding_sequence(rng, l2, consensi, shared, core=plen)
        pairs.append([s1, s2])
    return pairs


def multi_query(ref_len=1 << 24, nq=65_536, lo=100, hi=10_000, seed=SEED_BASE + 7):
    """One noncoding-like reference and ``nq`` query sequences of log-uniform
    length in [lo, hi]: every second query is a copy of a random reference
    window with 1-5 % substitutions (a read of the reference), the others are
    noncoding-like background with one planted exact reference piece of
    20-200 bases (clamped to the query).  Returns (ref, [queries])."""
    rng = _rng(seed)
    consensi = [random_bases(rng, 300) for _ in range(5)]
    ref, _ = noncoding_sequence(rng, ref_len, consensi, random_bases(rng, 0), 0)
    qs = []
    for i in range(nq):
        L = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        L = min(L, ref_len) if ref_len else L
        if i % 2 == 0 and ref_len >= L > 0:
            off = int(rng.integers(0, ref_len - L + 1))
            qs.append(mutate(rng, ref[off:off + L], float(rng.uniform(0.01, 0.05))))
        else:
            q, _ = noncoding_sequence(rng, L, consensi, random_bases(rng, 0), 0)
            plen = min(int(rng.integers(20, 201)), L, ref_len)
            if plen > 0:
                off = int(rng.integers(0, ref_len - plen + 1))
                _plant(rng, q, ref[off:off + plen].copy())
            qs.append(q)
    return ref, qs


def poisson_arrivals(rate, seconds, seed=SEED_BASE + 5):
    """Arrival times (seconds, ascending) of a Poisson process of ``rate``
    requests per second over [0, seconds): exponential gaps of mean 1/rate."""
    rng = _rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * seconds * 1.5) + 64)
    t = np.cumsum(gaps)
    return t[t < seconds]


def request_stream(count, pool_pair_lens, queries=16, seed=SEED_BASE + 6):
    """For ``count`` requests: the pool pair each one asks for (uniform over
    the pool) and ``queries`` follow-up (p, q) suffix pairs uniform over that
    pair's text of len1 + len2 + 2 symbols.  Returns (choice, P, Q) with P, Q
    int32 arrays of shape (count, queries)."""
    rng = _rng(seed)
    choice = rng.integers(0, len(pool_pair_lens), size=count)
    n = np.asarray([a + b + 2 for a, b in pool_pair_lens], dtype=np.int64)[choice]
    P = (rng.random((count, queries)) * n[:, None]).astype(np.int64).astype(np.int32)
    Q = (rng.random((count, queries)) * n[:, None]).astype(np.int64).astype(np.int32)
    return choice, P, Q


def fuzz_sequences(seed, nseq=2, max_len=64, alphabet=b"ACGT"):
    """Small random sequences for parity fuzzing; lengths uniform in
    [1, max_len], symbols uniform over ``alphabet``."""
    rng = _rng(seed)
    alpha = np.frombuffer(alphabet, dtype=np.uint8)
    out = []
    for _ in range(nseq):
        L = int(rng.integers(1, max_len + 1))
        out.append(alpha[rng.integers(0, alpha.size, size=L)])
    return out


def degenerate_cases():
    """Named degenerate inputs: single-symbol runs, period-2 strings, one-base
    sequences, no shared base, one sequence being a copy of the other."""
    A = lambda s: np.frombuffer(s, dtype=np.uint8).copy()
    return {
        "a_runs": [A(b"A" * 37), A(b"A" * 23)],
        "ac_period": [A(b"AC" * 20), A(b"CA" * 13)],
        "single_bases": [A(b"A"), A(b"A")],
        "one_base_each_diff": [A(b"A"), A(b"C")],
        "disjoint_alphabets": [A(b"ACACCA"), A(b"GTGGT")],
        "identical": [A(b"GATTACAGATTACA"), A(b"GATTACAGATTACA")],
        "prefix": [A(b"ACGTACGTTT"), A(b"ACGTAC")],
        "three_seqs": [A(b"ACGTTGCA"), A(b"TTGCAGG"), A(b"GGTTGCAT")],
    }
