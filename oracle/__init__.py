"""CPU oracle for the longest-overlap-region path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product library never
imports, loads or executes anything under ``oracle/``; the two share no code.

Everything here is the plain definition of what the method computes, written
out slowly (paper: "Solving The Longest Overlap Region Problem for Noncoding
DNA Sequences with GPU", arXiv 1404.3448):

* concatenation of several sequences into one text with unique separators
  (Section 3, "longest overlap prefix of two sequences"; the separator coding
  is this library's reading, the paper states none);
* suffix array by direct comparison sort (Section 3, Table 1);
* LCP array by direct comparison, lcp[0] = 0 (Section 3, LCP table);
* inverse suffix array / 1-based ranks (Section 3, Table 3);
* longest overlap region = maximum LCP over adjacent suffixes of different
  sequences, plus all positions of it (Section 3, lcp identity);
* LCP of arbitrary suffixes by direct comparison (Section 3, RMQ reduction);
* sparse table of range minima (the RMQ structure; Section 3 defines RMQ);
* the 1-bit split primitive and the radix sort built from it (Section 4,
  Algorithm 1) and the DC3 sample ranks / nonsample order (Section 3,
  Steps 1-2, Table 2);
* longest common substring by the O(n*m) dynamic program, a brute force that
  does not use suffix arrays, used to pin the overlap.

Heavy loops (suffix sort, LCP, DP) live in ``lor_oracle.c``; the rest is plain
numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lor_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblor_oracle.so")
_lib = None
_lock = threading.Lock()

# Symbol codes of the concatenated text (library reading; the paper fixes
# none): 0 is padding and never stored; the terminator of sequence i is
# nseq - i (so the last terminator is the smallest symbol); A, C, G, T follow
# as nseq+1 .. nseq+4, preserving A < C < G < T of Table 1.
BASES = b"ACGT"


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc; returns the library path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32p, u8p = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
            lib.oracle_suffix_array.argtypes = [u8p, i64, i32p, ctypes.c_int]
            lib.oracle_suffix_array.restype = ctypes.c_int
            lib.oracle_lcp_array.argtypes = [u8p, i64, i32p, i32p, ctypes.c_int]
            lib.oracle_lcp_array.restype = ctypes.c_int
            lib.oracle_check_suffix_array.argtypes = [u8p, i64, i32p, ctypes.c_int]
            lib.oracle_check_suffix_array.restype = ctypes.c_int64
            lib.oracle_lcp_pairs.argtypes = [u8p, i64, i32p, i32p, i64, i32p]
            lib.oracle_lcp_pairs.restype = ctypes.c_int
            vp = ctypes.c_void_p
            lib.oracle_check_suffix_array64.argtypes = [u8p, i64, vp, ctypes.c_int]
            lib.oracle_check_suffix_array64.restype = ctypes.c_int64
            lib.oracle_lcp_array64.argtypes = [u8p, i64, vp, i32p, ctypes.c_int]
            lib.oracle_lcp_array64.restype = ctypes.c_int
            lib.oracle_lcp_pairs64.argtypes = [u8p, i64, vp, vp, i64, vp]
            lib.oracle_lcp_pairs64.restype = ctypes.c_int
            lib.oracle_lcs_dp.argtypes = [u8p, i64, u8p, i64, u8p, u8p]
            lib.oracle_lcs_dp.restype = ctypes.c_int64
            lib.oracle_multi_query_one.argtypes = [u8p, i64, i32p, u8p, i64, ctypes.c_void_p]
            lib.oracle_multi_query_one.restype = ctypes.c_int
            _lib = lib
    return _lib


def _u8(a) -> np.ndarray:
    if isinstance(a, (bytes, bytearray)):
        a = np.frombuffer(bytes(a), dtype=np.uint8)
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


# --------------------------------------------------------------------------
# a1: encoding and concatenation
# --------------------------------------------------------------------------

def encode_concat(seqs):
    """Concatenate DNA sequences S_0 t_0 S_1 t_1 ... with unique terminators.

    Section 3 asks for the longest overlap of two (or more) sequences over one
    suffix array; the concatenation with separators is this library's reading.
    Returns (text uint8[n], seq_starts int64[nseq+1], sigma) where sigma is the
    number of symbol codes including the padding code 0.
    Raises ValueError on a symbol outside ACGT/acgt or on more than 250
    sequences (codes must fit in one byte).
    """
    seqs = [_u8(s) for s in seqs]
    nseq = len(seqs)
    if nseq < 1 or nseq > 250:
        raise ValueError("need 1..250 sequences")
    lut = np.full(256, 255, dtype=np.int32)
    for c, b in enumerate(BASES):
        lut[b] = nseq + 1 + c
        lut[ord(chr(b).lower())] = nseq + 1 + c
    parts, starts = [], [0]
    for i, s in enumerate(seqs):
        codes = lut[s]
        if codes.size and codes.max() == 255:
            raise ValueError(f"sequence {i} holds a symbol outside ACGT")
        parts.append(codes.astype(np.uint8))
        parts.append(np.array([nseq - i], dtype=np.uint8))
        starts.append(starts[-1] + len(s) + 1)
    text = np.concatenate(parts) if parts else np.zeros(0, np.uint8)
    return text, np.array(starts, dtype=np.int64), nseq + 5


def encode_raw(ascii_text):
    """Code one sequence without terminators: A=1, C=2, G=3, T=4.

    This is the setting of the worked example (Table 1: S = ATTGCTAC with
    eight suffixes and no terminator).  Returns (text, sigma=5).
    """
    s = _u8(ascii_text)
    lut = np.full(256, 255, dtype=np.int32)
    for c, b in enumerate(BASES):
        lut[b] = 1 + c
    codes = lut[s]
    if codes.size and codes.max() == 255:
        raise ValueError("symbol outside ACGT")
    return codes.astype(np.uint8), 5


# --------------------------------------------------------------------------
# a2..a8: suffix array (definition: sorted suffixes, Section 3, Table 1)
# --------------------------------------------------------------------------

def suffix_array(text, nthreads: int = 1) -> np.ndarray:
    t = _u8(text)
    sa = np.empty(t.size, dtype=np.int32)
    if _load().oracle_suffix_array(_ptr(t), t.size, _ptr(sa), int(nthreads)) != 0:
        raise MemoryError("oracle_suffix_array failed")
    return sa


def check_suffix_array(text, sa, nthreads: int = 1) -> int:
    """-1 if ``sa`` is the suffix array of ``text`` (permutation + every
    adjacent pair strictly increasing by direct comparison); otherwise the
    first rank where the definition fails (len(text) = not a permutation)."""
    t = _u8(text)
    s = np.ascontiguousarray(sa, dtype=np.int32)
    if s.size != t.size:
        return t.size
    return int(_load().oracle_check_suffix_array(_ptr(t), t.size, _ptr(s), int(nthreads)))


def inverse_suffix_array(sa) -> np.ndarray:
    """isa[sa[k]] = k (0-based ranks; Table 3 prints them 1-based)."""
    sa = np.asarray(sa)
    isa = np.empty(sa.size, dtype=np.int32)
    isa[sa] = np.arange(sa.size, dtype=np.int32)
    return isa


def sample_ranks(text) -> np.ndarray:
    """DC3 Step 1 result (Section 3, Table 2): for i with i mod 3 != 0, the
    1-based rank of suffix i among the sample suffixes; 0 (printed as the
    undefined symbol) for i mod 3 == 0."""
    sa = suffix_array(text)
    out = np.zeros(len(sa), dtype=np.int32)
    r = 0
    for p in sa:
        if p % 3 != 0:
            r += 1
            out[p] = r
    return out


def nonsample_order(text) -> np.ndarray:
    """DC3 Step 2 result (Section 3): positions i mod 3 == 0 in suffix order."""
    sa = suffix_array(text)
    return sa[sa % 3 == 0].astype(np.int32)


# --------------------------------------------------------------------------
# a9: LCP array (Section 3, LCP table: lcp[0] = 0)
# --------------------------------------------------------------------------

def lcp_array(text, sa, nthreads: int = 1) -> np.ndarray:
    t = _u8(text)
    s = np.ascontiguousarray(sa, dtype=np.int32)
    lcp = np.empty(t.size, dtype=np.int32)
    if _load().oracle_lcp_array(_ptr(t), t.size, _ptr(s), _ptr(lcp), int(nthreads)) != 0:
        raise ValueError("oracle_lcp_array failed")
    return lcp


# --------------------------------------------------------------------------
# a10: longest overlap region and all of its positions
# --------------------------------------------------------------------------

def seq_of(positions, seq_starts) -> np.ndarray:
    """Index of the sequence a text position belongs to (a terminator belongs
    to the sequence it closes)."""
    return (np.searchsorted(np.asarray(seq_starts), np.asarray(positions), side="right") - 1
            ).astype(np.int64)


def longest_overlap(text, sa, lcp, seq_starts):
    """Longest overlap region over adjacent suffixes of different sequences.

    Section 3: the LCP of two suffixes is the minimum of the adjacent LCPs
    between them, so the longest region shared by two sequences is the largest
    LCP between rank-adjacent suffixes that start in different sequences.
    Readings (the paper is silent): ``rank`` is the smallest rank k attaining
    the maximum; seq_a/pos_a is the suffix of the lower sequence id at ranks
    k-1, k; ``positions`` lists every text position p whose length-L prefix
    also occurs in another sequence, i.e. every member of a maximal rank run
    with adjacent LCP >= L that holds suffixes of two or more sequences,
    sorted ascending.  L == 0 gives rank = seq = pos = -1 and no positions.
    """
    sa = np.asarray(sa, dtype=np.int64)
    lcp = np.asarray(lcp, dtype=np.int64)
    n = sa.size
    res = dict(length=0, rank=-1, seq_a=-1, pos_a=-1, seq_b=-1, pos_b=-1,
               positions=np.zeros(0, dtype=np.int64))
    if n < 2:
        return res
    sq = seq_of(sa, seq_starts)
    cross = np.zeros(n, dtype=bool)
    cross[1:] = sq[1:] != sq[:-1]
    cand = np.where(cross, lcp, -1)
    L = int(cand.max())
    if L <= 0:
        return res
    k = int(np.argmax(cand == L))
    a, b = int(sa[k - 1]), int(sa[k])
    sa_, sb_ = int(sq[k - 1]), int(sq[k])
    if sa_ > sb_:
        a, b, sa_, sb_ = b, a, sb_, sa_
    starts = np.asarray(seq_starts, dtype=np.int64)
    res.update(length=L, rank=k, seq_a=sa_, pos_a=a - int(starts[sa_]),
               seq_b=sb_, pos_b=b - int(starts[sb_]))
    run_start = np.ones(n, dtype=bool)
    run_start[1:] = lcp[1:] < L
    run_id = np.cumsum(run_start) - 1
    qual = np.zeros(int(run_id[-1]) + 1, dtype=bool)
    seeds = (~run_start) & cross
    qual[run_id[seeds]] = True
    members = sa[qual[run_id]]
    res["positions"] = np.sort(members)
    return res


def lcs_dp(a, b, with_positions: bool = True):
    """Longest common substring of two ASCII sequences by the O(n*m) dynamic
    program (brute force; no suffix array).  Returns (L, starts_a, starts_b):
    the start offsets of every occurrence of a length-L common substring."""
    a, b = _u8(a), _u8(b)
    ma = np.zeros(max(a.size, 1), dtype=np.uint8)
    mb = np.zeros(max(b.size, 1), dtype=np.uint8)
    L = _load().oracle_lcs_dp(_ptr(a), a.size, _ptr(b), b.size,
                              _ptr(ma) if with_positions else None,
                              _ptr(mb) if with_positions else None)
    if L < 0:
        raise MemoryError("oracle_lcs_dp failed")
    return int(L), np.flatnonzero(ma[:a.size]), np.flatnonzero(mb[:b.size])


def overlap_by_dp(seqs):
    """Overlap length and position set over several sequences by pairwise DP:
    L = max over pairs of the longest common substring; a text position is in
    the set when its length-L substring also occurs in another sequence."""
    seqs = [_u8(s) for s in seqs]
    best = 0
    pair_res = {}
    for i in range(len(seqs)):
        for j in range(i + 1, len(seqs)):
            r = lcs_dp(seqs[i], seqs[j])
            pair_res[(i, j)] = r
            best = max(best, r[0])
    starts = np.cumsum([0] + [len(s) + 1 for s in seqs])
    pos = set()
    if best > 0:
        for (i, j), (L, pa, pb) in pair_res.items():
            if L == best:
                pos.update(int(starts[i] + x) for x in pa)
                pos.update(int(starts[j] + x) for x in pb)
    return best, np.array(sorted(pos), dtype=np.int64)


# --------------------------------------------------------------------------
# a11..a12: sparse table and LCP queries between arbitrary suffixes
# --------------------------------------------------------------------------

def sparse_table_levels(n: int) -> int:
    """floor(log2 n) + 1 levels (level j covers windows of 2**j entries)."""
    return max(1, int(n).bit_length()) if n > 0 else 1


def sparse_table(lcp) -> np.ndarray:
    """ST[j][i] = min(lcp[i : min(i + 2**j, n)]) (range minima over windows
    clipped at the end of the array), built level by level:
    ST[j][i] = min(ST[j-1][i], ST[j-1][i + 2**(j-1)]) where that index exists."""
    lcp = np.asarray(lcp, dtype=np.int32)
    n = lcp.size
    J = sparse_table_levels(n)
    st = np.empty((J, n), dtype=np.int32)
    st[0] = lcp
    for j in range(1, J):
        h = 1 << (j - 1)
        st[j] = st[j - 1]
        if h < n:
            st[j, : n - h] = np.minimum(st[j - 1, : n - h], st[j - 1, h:])
    return st


def block_minima(lcp, block: int = 32) -> np.ndarray:
    """min(lcp[b*block : min((b+1)*block, n)]) for every block b (the blocks
    of the linear-space range-minimum structure; Section 3 RMQ)."""
    lcp = np.asarray(lcp, dtype=np.int32)
    n = lcp.size
    nb = -(-n // block)
    return np.array([lcp[b * block:min((b + 1) * block, n)].min() for b in range(nb)], dtype=np.int32)


def block_sparse_table(lcp, block: int = 32) -> np.ndarray:
    """The sparse table over the block minima (rows as in sparse_table)."""
    return sparse_table(block_minima(lcp, block))


def rmq_argmin(lcp, isa, p, q):
    """Section 3, RMQ returning the index: for suffixes p != q with ranks
    r1 < r2, (min(lcp[r1+1 .. r2]), the leftmost rank k in (r1, r2] holding
    it); p == q gives (n - p, -1).  By definition, one query at a time."""
    lcp = np.asarray(lcp)
    n = lcp.size
    val = np.empty(len(p), dtype=np.int32)
    arg = np.empty(len(p), dtype=np.int32)
    for i, (a, b) in enumerate(zip(p, q)):
        if a == b:
            val[i], arg[i] = n - a, -1
            continue
        r1, r2 = sorted((int(isa[a]), int(isa[b])))
        w = lcp[r1 + 1:r2 + 1]
        j = int(np.argmin(w))  # first occurrence of the minimum
        val[i], arg[i] = w[j], r1 + 1 + j
    return val, arg


def topk_overlaps(text, sa, lcp, seq_starts, K):
    """The K largest left-maximal cross-sequence adjacent pairs by (LCP desc,
    rank asc), by definition over every rank: candidates are ranks k >= 1
    with SA[k-1], SA[k] in different sequences, LCP[k] > 0, and a or b = 0 or
    text[a-1] != text[b-1].  Returns records like longest_overlap's (without
    positions), largest first."""
    t = _u8(text)
    sa = np.asarray(sa)
    lcp = np.asarray(lcp)
    seq = seq_of(sa, seq_starts)
    cand = []
    for k in range(1, t.size):
        a, b = int(sa[k - 1]), int(sa[k])
        if lcp[k] <= 0 or seq[k - 1] == seq[k]:
            continue
        if a != 0 and b != 0 and t[a - 1] == t[b - 1]:
            continue
        cand.append((-int(lcp[k]), k))
    cand.sort()
    out = []
    starts = np.asarray(seq_starts)
    for negl, k in cand[:K]:
        a, b = int(sa[k - 1]), int(sa[k])
        qa, qb = int(seq[k - 1]), int(seq[k])
        if qa > qb:
            a, b, qa, qb = b, a, qb, qa
        out.append(dict(length=-negl, rank=k, seq_a=qa, pos_a=a - int(starts[qa]), seq_b=qb,
                        pos_b=b - int(starts[qb])))
    return out


def multi_query(ref, queries):
    """One reference against many queries (uppercase ASCII): per query (L, q, r) with L the
    length of the longest substring it shares with the reference, q the
    smallest query offset where a length-L shared substring starts and r the
    smallest reference offset of that substring ((0, -1, -1) when L = 0).
    Works on the ASCII bases; the reference's suffixes are sorted once
    (plain merge sort) and every query suffix is matched by binary search
    with direct comparison."""
    r = _u8(ref)
    sa_r = suffix_array(r) if r.size else np.zeros(0, np.int32)
    out = np.empty((len(queries), 3), dtype=np.int64)
    res = np.empty(3, dtype=np.int64)
    for i, qs in enumerate(queries):
        q = _u8(qs)
        _load().oracle_multi_query_one(_ptr(r), r.size, _ptr(sa_r), _ptr(q), q.size, _ptr(res))
        out[i] = res
    return out


def lcp_pairs(text, p, q) -> np.ndarray:
    """LCP of suffixes p[i] and q[i] by direct symbol comparison; the LCP of a
    suffix with itself is its length (Section 3, lcp of arbitrary suffixes)."""
    t = _u8(text)
    p = np.ascontiguousarray(p, dtype=np.int32)
    q = np.ascontiguousarray(q, dtype=np.int32)
    out = np.empty(p.size, dtype=np.int32)
    if _load().oracle_lcp_pairs(_ptr(t), t.size, _ptr(p), _ptr(q), p.size, _ptr(out)) != 0:
        raise ValueError("query position out of range")
    return out


# --------------------------------------------------------------------------
# the same definitions with int64 indices (texts past 2^31 symbols)
# --------------------------------------------------------------------------

def check_suffix_array64(text, sa, nthreads: int = 1) -> int:
    """check_suffix_array for an int64 suffix array."""
    t = _u8(text)
    s = np.ascontiguousarray(sa, dtype=np.int64)
    if s.size != t.size:
        return t.size
    return int(_load().oracle_check_suffix_array64(_ptr(t), t.size, s.ctypes.data, int(nthreads)))


def lcp_array64(text, sa, nthreads: int = 1) -> np.ndarray:
    """lcp_array for an int64 suffix array (int32 values; ValueError when one
    does not fit)."""
    t = _u8(text)
    s = np.ascontiguousarray(sa, dtype=np.int64)
    lcp = np.empty(t.size, dtype=np.int32)
    if _load().oracle_lcp_array64(_ptr(t), t.size, s.ctypes.data, _ptr(lcp), int(nthreads)) != 0:
        raise ValueError("oracle_lcp_array64 failed")
    return lcp


def lcp_pairs64(text, p, q) -> np.ndarray:
    """lcp_pairs with int64 positions and answers."""
    t = _u8(text)
    p = np.ascontiguousarray(p, dtype=np.int64)
    q = np.ascontiguousarray(q, dtype=np.int64)
    out = np.empty(p.size, dtype=np.int64)
    if _load().oracle_lcp_pairs64(_ptr(t), t.size, p.ctypes.data, q.ctypes.data, p.size, out.ctypes.data) != 0:
        raise ValueError("query position out of range")
    return out


def overlap_max_scan(sa, lcp, seq_starts, chunk: int = 1 << 24):
    """(L, k) of longest_overlap -- the largest LCP between rank-adjacent
    suffixes of different sequences and the smallest rank attaining it
    (Section 3) -- scanned over ranks in chunks, so that arrays of billions of
    entries need no whole-array temporaries.  (0, -1) when no such pair shares
    a symbol."""
    sa = np.asarray(sa)
    lcp = np.asarray(lcp)
    n = sa.size
    best, best_k = 0, -1
    for lo in range(1, n, chunk):
        hi = min(n, lo + chunk)
        sq = seq_of(sa[lo - 1:hi], seq_starts)
        cross = sq[1:] != sq[:-1]
        cand = np.where(cross, lcp[lo:hi].astype(np.int64), -1)
        m = int(cand.max())
        if m > best:
            best, best_k = m, lo + int(np.argmax(cand == m))
    return best, best_k


def longest_overlap_large(text, sa, lcp, seq_starts):
    """longest_overlap for texts of billions of symbols.  L and k come from
    overlap_max_scan; the positions are those of longest_overlap applied to
    the ranks that can hold them: every maximal run of ranks with adjacent
    LCP >= L (LCP set to 0 at each run's first rank, so that runs stay
    apart), which is where longest_overlap finds its qualifying runs."""
    lcp = np.asarray(lcp)
    sa = np.asarray(sa)
    L, k = overlap_max_scan(sa, lcp, seq_starts)
    res = dict(length=0, rank=-1, seq_a=-1, pos_a=-1, seq_b=-1, pos_b=-1,
               positions=np.zeros(0, dtype=np.int64))
    if L <= 0:
        return res
    hits = np.flatnonzero(lcp >= L)
    hits = hits[hits >= 1]
    ranks = np.unique(np.concatenate([hits - 1, hits]))
    sub_lcp = lcp[ranks].astype(np.int64)
    first = np.ones(ranks.size, dtype=bool)
    first[1:] = ranks[1:] != ranks[:-1] + 1
    first |= sub_lcp < L
    sub_lcp[first] = 0
    sub = longest_overlap(text, sa[ranks], sub_lcp, seq_starts)
    starts = np.asarray(seq_starts, dtype=np.int64)
    a, b = int(sa[k - 1]), int(sa[k])
    qa, qb = (int(x) for x in seq_of(np.array([a, b]), starts))
    if qa > qb:
        a, b, qa, qb = b, a, qb, qa
    res.update(length=L, rank=k, seq_a=qa, pos_a=a - int(starts[qa]), seq_b=qb, pos_b=b - int(starts[qb]),
               positions=sub["positions"])
    return res


# --------------------------------------------------------------------------
# Section 4: the 1-bit split primitive and the radix sort built from it
# --------------------------------------------------------------------------

def split_1bit(keys, bit: int):
    """One split step of Section 4 (Algorithm 1): b = bit of each key,
    e = NOT b, f = exclusive prefix sum of e, totalFalse = e[n-1] + f[n-1],
    destination = b ? i - f + totalFalse : f.  Returns (out, e, f, total)."""
    keys = np.asarray(keys, dtype=np.uint64)
    n = keys.size
    b = ((keys >> np.uint64(bit)) & np.uint64(1)).astype(np.int64)
    e = 1 - b
    f = np.zeros(n, dtype=np.int64)
    if n > 1:
        f[1:] = np.cumsum(e)[:-1]
    total = int(e[-1] + f[-1]) if n else 0
    i = np.arange(n, dtype=np.int64)
    dest = np.where(b == 1, i - f + total, f)
    out = np.empty_like(keys)
    out[dest] = keys
    return out, e, f, total


def radix_sort_split(keys, nbits: int, values=None):
    """LSD radix sort by repeated 1-bit splits over bits 0..nbits-1
    (Section 4, Algorithm 1).  Stable; returns (keys, values)."""
    keys = np.asarray(keys, dtype=np.uint64)
    vals = np.arange(keys.size, dtype=np.int64) if values is None else np.asarray(values)
    for bit in range(nbits):
        b = ((keys >> np.uint64(bit)) & np.uint64(1)).astype(np.int64)
        e = 1 - b
        f = np.zeros(keys.size, dtype=np.int64)
        if keys.size > 1:
            f[1:] = np.cumsum(e)[:-1]
        total = int(e[-1] + f[-1]) if keys.size else 0
        i = np.arange(keys.size, dtype=np.int64)
        dest = np.where(b == 1, i - f + total, f)
        nk = np.empty_like(keys)
        nv = np.empty_like(vals)
        nk[dest] = keys
        nv[dest] = vals
        keys, vals = nk, nv
    return keys, vals


# --------------------------------------------------------------------------
# many independent pairs (the batched and served workloads): the functions
# above, once per pair, spread over host processes
# --------------------------------------------------------------------------

def pair_overlap(a, b, queries=None):
    """Record and positions of one pair alone (its own text S1#S2$), and the
    direct-comparison LCP of each (p, q) suffix pair of that text when
    ``queries`` = (P, Q) is given."""
    text, starts, _ = encode_concat([a, b])
    sa = suffix_array(text)
    lcp = lcp_array(text, sa)
    ov = longest_overlap(text, sa, lcp, starts)
    if queries is not None:
        ov["answers"] = lcp_pairs(text, np.asarray(queries[0], np.int32), np.asarray(queries[1], np.int32))
    return ov


def _pair_overlap_chunk(items):
    return [pair_overlap(a, b, q) for a, b, q in items]


def pair_overlaps(pairs, queries=None, processes=None):
    """pair_overlap for every pair, in ``processes`` spawned worker processes
    (default: every host core).  Spawned, not forked, so that a caller
    holding a CUDA context can use it.  Returns the records in pair order."""
    import multiprocessing as mp
    items = [(a, b, None if queries is None else queries[i]) for i, (a, b) in enumerate(pairs)]
    procs = processes or os.cpu_count() or 1
    if procs <= 1 or len(items) < 2:
        return _pair_overlap_chunk(items)
    build()
    # interleaved chunks balance long and short pairs across the workers
    nchunk = min(len(items), procs * 4)
    chunks = [items[c::nchunk] for c in range(nchunk)]
    with mp.get_context("spawn").Pool(min(procs, nchunk)) as pool:
        res = pool.map(_pair_overlap_chunk, chunks)
    out = [None] * len(items)
    for c, r in enumerate(res):
        out[c::nchunk] = r
    return out
