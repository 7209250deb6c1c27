"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test ties an oracle function to something other than itself: values the
paper prints for its worked example (tests/golden/), closed forms, a theorem
(the LCP identity of Section 3), an independent brute force (the O(n*m)
longest-common-substring dynamic program; Python string comparison), or
planted structure.  Chosen so that a dropped term, wrong sign, wrong index or
transposed operand in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

from golden.load import load
import lor_inputs as gen


# ---------------------------------------------------------------- paper example

@pytest.fixture(scope="module")
def paper(oracle_mod):
    g = load("paper_example.txt")
    text, sigma = oracle_mod.encode_raw(g["text"][0].encode())
    return g, text


def test_table1_suffix_array(oracle_mod, paper):
    g, text = paper
    assert oracle_mod.suffix_array(text).tolist() == g["sa"]


def test_table3_ranks(oracle_mod, paper):
    g, text = paper
    isa = oracle_mod.inverse_suffix_array(oracle_mod.suffix_array(text))
    assert (isa + 1).tolist() == g["ranks1"]


def test_table2_sample_ranks(oracle_mod, paper):
    g, text = paper
    n = len(text)
    assert [i for i in range(n) if i % 3 != 0] == g["sample_set"]
    assert [i for i in range(n) if i % 3 == 1] == g["b1"]
    assert [i for i in range(n) if i % 3 == 2] == g["b2"]
    assert oracle_mod.sample_ranks(text).tolist() == g["sample_ranks"]


def test_step2_nonsample_order(oracle_mod, paper):
    g, text = paper
    order = oracle_mod.nonsample_order(text).tolist()
    assert order == g["nonsample_order"]
    ranks = oracle_mod.sample_ranks(text)
    pairs = [v for i in order for v in (int(text[i]), int(ranks[i + 1]))]
    assert pairs == g["nonsample_pairs"]
    # the pairs themselves are in increasing lexicographic order
    tup = list(zip(pairs[0::2], pairs[1::2]))
    assert tup == sorted(tup)


def test_lcp_table(oracle_mod, paper):
    g, text = paper
    sa = oracle_mod.suffix_array(text)
    assert oracle_mod.lcp_array(text, sa).tolist() == g["lcp"]


# ---------------------------------------------------------------- split / radix

def test_split_example(oracle_mod):
    g = load("split_example.txt")
    out, e, f, total = oracle_mod.split_1bit(g["keys"], g["bit"][0])
    bits = [(k >> g["bit"][0]) & 1 for k in g["keys"]]
    assert bits == g["L"]
    assert e.tolist() == g["E"]
    assert f.tolist() == g["F"]
    assert total == g["total_false"][0]
    assert out.tolist() == g["out"]


def test_radix_split_sort_matches_builtin_sort(oracle_mod):
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 12, size=3000, dtype=np.uint64)
    k, v = oracle_mod.radix_sort_split(keys, 12)
    ref = sorted(range(len(keys)), key=lambda i: (int(keys[i]), i))   # stable
    assert v.tolist() == ref
    assert k.tolist() == [int(keys[i]) for i in ref]


def test_radix_split_sort_partial_bits_is_stable_on_low_bits(oracle_mod):
    rng = np.random.default_rng(8)
    keys = rng.integers(0, 1 << 16, size=2000, dtype=np.uint64)
    _, v = oracle_mod.radix_sort_split(keys, 5)
    ref = sorted(range(len(keys)), key=lambda i: (int(keys[i]) & 31, i))
    assert v.tolist() == ref


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("k", [1, 2, 3, 7, 50, 301])
def test_single_symbol_run_closed_form(oracle_mod, k):
    text, _ = oracle_mod.encode_raw(b"A" * k)
    sa = oracle_mod.suffix_array(text)
    assert sa.tolist() == list(range(k - 1, -1, -1))
    assert oracle_mod.lcp_array(text, sa).tolist() == list(range(k))


@pytest.mark.parametrize("k", [1, 2, 5, 40])
def test_period_two_closed_form(oracle_mod, k):
    text, _ = oracle_mod.encode_raw(b"AC" * k)
    sa = oracle_mod.suffix_array(text)
    a_part = list(range(2 * k - 2, -1, -2))
    c_part = list(range(2 * k - 1, 0, -2))
    assert sa.tolist() == a_part + c_part
    lcp = oracle_mod.lcp_array(text, sa).tolist()
    assert lcp == [0] + list(range(2, 2 * k - 1, 2)) + [0] + list(range(1, 2 * k - 2, 2))


# ---------------------------------------------------------------- brute force

def test_all_short_strings_against_python_string_order(oracle_mod):
    alpha = "ACGT"
    for L in range(1, 7):
        for tup in itertools.product(alpha, repeat=L):
            s = "".join(tup)
            text, _ = oracle_mod.encode_raw(s.encode())
            sa = oracle_mod.suffix_array(text).tolist()
            ref = sorted(range(L), key=lambda i: s[i:])
            assert sa == ref, s
            lcp = oracle_mod.lcp_array(text, np.array(sa, np.int32)).tolist()
            ref_lcp = [0] + [len(os.path.commonprefix([s[ref[k - 1]:], s[ref[k]:]]))
                             for k in range(1, L)]
            assert lcp == ref_lcp, s


def test_terminated_text_order(oracle_mod):
    # Separator codes sit below every base and the last terminator is the
    # smallest symbol, so SA[0] = n-1 and SA[1] = |S1| for two sequences.
    seqs = [np.frombuffer(b"GATTACA", np.uint8), np.frombuffer(b"TAGACAT", np.uint8)]
    text, starts, sigma = oracle_mod.encode_concat(seqs)
    assert sigma == 7
    assert text.tolist() == [5, 3, 6, 6, 3, 4, 3, 2, 6, 3, 5, 3, 4, 3, 6, 1]
    sa = oracle_mod.suffix_array(text)
    assert sa[0] == len(text) - 1 and sa[1] == 7
    assert oracle_mod.check_suffix_array(text, sa) == -1


def test_check_suffix_array_rejects_wrong_arrays(oracle_mod):
    seqs, _ = gen.pair_uniform(n_each=500, plant_len=40, seed=3)
    text, _, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text)
    assert oracle_mod.check_suffix_array(text, sa, nthreads=3) == -1
    bad = sa.copy()
    bad[10], bad[11] = bad[11], bad[10]
    assert oracle_mod.check_suffix_array(text, bad) == 11
    dup = sa.copy()
    dup[5] = dup[6]
    assert oracle_mod.check_suffix_array(text, dup) == len(text)


def test_parallel_sort_equals_serial(oracle_mod):
    seqs, _ = gen.pair_noncoding(n_each=20_000, seed=11, shared_len=3000, core=600)
    text, _, _ = oracle_mod.encode_concat(seqs)
    a = oracle_mod.suffix_array(text, nthreads=1)
    b = oracle_mod.suffix_array(text, nthreads=8)
    assert np.array_equal(a, b)
    assert oracle_mod.check_suffix_array(text, a) == -1
    assert np.array_equal(oracle_mod.lcp_array(text, a, 1), oracle_mod.lcp_array(text, a, 5))


# ---------------------------------------------------------------- LCP identity

def test_lcp_identity_of_section3(oracle_mod):
    # lcp(S_SA[i], S_SA[j]) = min over i < k <= j of lcp[k]   (Section 3)
    rng = np.random.default_rng(5)
    for trial in range(30):
        seqs = gen.fuzz_sequences(100 + trial, nseq=2, max_len=80,
                                  alphabet=b"AC" if trial % 2 else b"ACGT")
        text, _, _ = oracle_mod.encode_concat(seqs)
        n = len(text)
        sa = oracle_mod.suffix_array(text)
        lcp = oracle_mod.lcp_array(text, sa)
        isa = oracle_mod.inverse_suffix_array(sa)
        p = rng.integers(0, n, 200).astype(np.int32)
        q = rng.integers(0, n, 200).astype(np.int32)
        got = oracle_mod.lcp_pairs(text, p, q)
        for a, b, g in zip(p, q, got):
            if a == b:
                assert g == n - a
            else:
                r1, r2 = sorted((isa[a], isa[b]))
                assert g == lcp[r1 + 1:r2 + 1].min()


# ---------------------------------------------------------------- sparse table

def test_sparse_table_is_window_minimum(oracle_mod):
    rng = np.random.default_rng(9)
    for n in [1, 2, 3, 7, 64, 100, 257]:
        lcp = rng.integers(0, 20, n).astype(np.int32)
        st = oracle_mod.sparse_table(lcp)
        assert st.shape == (oracle_mod.sparse_table_levels(n), n)
        for j in range(st.shape[0]):
            for i in range(n):
                assert st[j, i] == lcp[i:min(i + (1 << j), n)].min()


def test_block_table_windows_are_ranges_of_the_lcp_array(oracle_mod):
    """Entry (j, b) of the block table is the minimum of the LCP entries of
    blocks b .. b + 2^j - 1 (clipped at n), by brute force on small arrays;
    and the minimum of any rank range split into partial blocks and whole
    blocks equals the range minimum (the query rule of the linear-space RMQ)."""
    rng = np.random.default_rng(10)
    for n in [1, 31, 32, 33, 64, 100, 1000]:
        lcp = rng.integers(0, 50, n).astype(np.int32)
        bt = oracle_mod.block_sparse_table(lcp)
        nb = -(-n // 32)
        assert bt.shape == (oracle_mod.sparse_table_levels(nb), nb)
        for j in range(bt.shape[0]):
            for b in range(nb):
                assert bt[j, b] == lcp[b * 32:min((b + (1 << j)) * 32, n)].min()
        for _ in range(200):
            a, e = sorted(int(x) for x in rng.integers(0, n, 2))
            ba, bb = a // 32, e // 32
            if ba == bb:
                m = lcp[a:e + 1].min()
            else:
                m = min(lcp[a:(ba + 1) * 32].min(), lcp[bb * 32:e + 1].min())
                if bb - ba - 1 > 0:
                    j = (bb - ba - 1).bit_length() - 1
                    m = min(m, bt[j, ba + 1], bt[j, bb - (1 << j)])
            assert m == lcp[a:e + 1].min()


def test_rmq_argmin_is_the_leftmost_minimum_and_the_suffix_lcp(oracle_mod):
    """The index form of the RMQ: the value is the LCP of the two suffixes by
    direct comparison (Section 3's identity), and the index is the first rank
    of the range that holds it."""
    rng = np.random.default_rng(11)
    for alpha in [b"AC", b"A", b"ACGT"]:
        a = np.frombuffer(alpha, np.uint8)
        seqs = [a[rng.integers(0, a.size, 40)], a[rng.integers(0, a.size, 25)]]
        text, _, _ = oracle_mod.encode_concat(seqs)
        n = text.size
        sa = oracle_mod.suffix_array(text)
        lcp = oracle_mod.lcp_array(text, sa)
        isa = oracle_mod.inverse_suffix_array(sa)
        pp, qq = np.meshgrid(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32))
        p, q = pp.ravel(), qq.ravel()
        val, arg = oracle_mod.rmq_argmin(lcp, isa, p, q)
        np.testing.assert_array_equal(val, oracle_mod.lcp_pairs(text, p, q))
        for i in range(p.size):
            if p[i] == q[i]:
                assert arg[i] == -1
                continue
            r1, r2 = sorted((isa[p[i]], isa[q[i]]))
            assert r1 < arg[i] <= r2 and lcp[arg[i]] == val[i]
            assert (lcp[r1 + 1:arg[i]] > val[i]).all()


def test_multi_query_oracle_against_the_dp(oracle_mod):
    """One reference against many queries: the length is the DP's longest
    common substring, the query offset the smallest DP start in the query,
    the reference offset the first occurrence of that substring (bytes.find),
    on random, repetitive and degenerate cases."""
    rng = np.random.default_rng(12)
    A = np.frombuffer(b"ACGT", np.uint8)
    refs = [A[rng.integers(0, 4, 400)], np.frombuffer(b"ACACACACACACAC" * 8, np.uint8),
            np.frombuffer(b"A", np.uint8), np.zeros(0, np.uint8)]
    for ref in refs:
        qs = [A[rng.integers(0, 4, int(rng.integers(0, 50)))] for _ in range(25)]
        qs += [np.frombuffer(b"CA" * 7, np.uint8), np.zeros(0, np.uint8), np.frombuffer(b"T", np.uint8)]
        if ref.size > 60:
            qs.append(ref[17:60].copy())
        res = oracle_mod.multi_query(ref, qs)
        for q, (L, qq, rr) in zip(qs, res):
            Ld, _, sb = oracle_mod.lcs_dp(ref, q) if len(q) and len(ref) else (0, [], [])
            if Ld == 0:
                assert (L, qq, rr) == (0, -1, -1)
                continue
            eq = int(min(sb))
            assert (L, qq, rr) == (Ld, eq, bytes(ref).find(bytes(q[eq:eq + Ld])))


def test_topk_overlaps_first_is_the_longest_overlap_and_entries_are_maximal(oracle_mod):
    """The largest left-maximal cross pair is the longest overlap (a pair at
    the maximum is always left-maximal: one more equal symbol on the left
    would give a longer cross overlap), so the first top-k entry equals
    longest_overlap's record and its length the DP's; every entry is a cross
    pair, left-maximal, with the length of the direct common prefix, in
    (length desc, rank asc) order."""
    rng = np.random.default_rng(13)
    A = np.frombuffer(b"ACGT", np.uint8)
    for trial in range(40):
        alpha = [A, A[:2], A[:1]][trial % 3]
        seqs = [alpha[rng.integers(0, alpha.size, int(rng.integers(1, 60)))] for _ in range(2 + trial % 3)]
        text, starts, _ = oracle_mod.encode_concat(seqs)
        sa = oracle_mod.suffix_array(text)
        lcp = oracle_mod.lcp_array(text, sa)
        ov = oracle_mod.longest_overlap(text, sa, lcp, starts)
        top = oracle_mod.topk_overlaps(text, sa, lcp, starts, 50)
        if ov["length"] == 0:
            assert top == []
            continue
        assert {k: top[0][k] for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b")} == \
            {k: ov[k] for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b")}
        assert top[0]["length"] == oracle_mod.overlap_by_dp(seqs)[0]
        prev = None
        for e in top:
            a = int(starts[e["seq_a"]]) + e["pos_a"]
            b = int(starts[e["seq_b"]]) + e["pos_b"]
            assert e["seq_a"] < e["seq_b"]
            assert a == 0 or b == 0 or text[a - 1] != text[b - 1]
            assert e["length"] == oracle_mod.lcp_pairs(text, np.array([a], np.int32), np.array([b], np.int32))[0]
            assert sorted((sa[e["rank"] - 1], sa[e["rank"]])) == sorted((a, b))
            key = (-e["length"], e["rank"])
            assert prev is None or key > prev
            prev = key


def _brute_topk(text, starts, nseq):
    """Every cross-sequence left-maximal adjacent pair, by brute force: the
    suffixes sorted as Python byte strings, the common prefix of each adjacent
    pair counted symbol by symbol, the sequence of a position found by walking
    the start offsets, the left symbols compared directly."""
    t = bytes(np.asarray(text, np.uint8))
    n = len(t)
    order = sorted(range(n), key=lambda i: t[i:])
    st = [int(x) for x in starts]

    def seq(p):
        q = 0
        while q + 1 < len(st) and st[q + 1] <= p:
            q += 1
        return q

    out = []
    for k in range(1, n):
        a, b = order[k - 1], order[k]
        h = 0
        while a + h < n and b + h < n and t[a + h] == t[b + h]:
            h += 1
        if h == 0 or seq(a) == seq(b):
            continue
        if a > 0 and b > 0 and t[a - 1] == t[b - 1]:
            continue
        qa, qb, pa, pb = seq(a), seq(b), a, b
        if qa > qb:
            qa, qb, pa, pb = qb, qa, pb, pa
        out.append(dict(length=h, rank=k, seq_a=qa, pos_a=pa - st[qa], seq_b=qb, pos_b=pb - st[qb]))
    out.sort(key=lambda e: (-e["length"], e["rank"]))
    return out


def test_topk_overlaps_is_complete_against_brute_force(oracle_mod):
    """With K at least the number of candidates, topk_overlaps returns exactly
    the set of cross-sequence left-maximal adjacent pairs (Section 3: the LCP
    of adjacent suffixes from two different sequences, the longest overlap
    being the largest), enumerated here by brute force, in (length desc, rank
    asc) order; a smaller K returns a prefix of that list.  A skip rule that
    drops a lesser candidate, or keeps a pair that is not left-maximal, fails
    here."""
    rng = np.random.default_rng(29)
    A = np.frombuffer(b"ACGT", np.uint8)
    cases = 0
    for trial in range(60):
        alpha = [A, A[:2], A[:1], A[:3]][trial % 4]
        nseq = 2 + trial % 3
        seqs = [alpha[rng.integers(0, alpha.size, int(rng.integers(1, 40)))] for _ in range(nseq)]
        text, starts, _ = oracle_mod.encode_concat(seqs)
        sa = oracle_mod.suffix_array(text)
        lcp = oracle_mod.lcp_array(text, sa)
        want = _brute_topk(text, starts, nseq)
        got = oracle_mod.topk_overlaps(text, sa, lcp, starts, len(text) + 1)
        assert got == want
        for K in (0, 1, 2, max(1, len(want) // 2), len(want)):
            assert oracle_mod.topk_overlaps(text, sa, lcp, starts, K) == want[:K]
        cases += len(want) > 2
    assert cases > 20  # most cases have more than the single longest pair
    # a case with several pairs of one length, where only the rank orders them
    seqs = [np.frombuffer(b"ACGTACGA", np.uint8), np.frombuffer(b"CGTTACGC", np.uint8)]
    text, starts, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text)
    lcp = oracle_mod.lcp_array(text, sa)
    assert oracle_mod.topk_overlaps(text, sa, lcp, starts, 100) == _brute_topk(text, starts, 2)


# ---------------------------------------------------------------- LCS DP pins

def _brute_lcs(a: bytes, b: bytes):
    best, sa_, sb_ = 0, set(), set()
    subs_b = {}
    for j in range(len(b)):
        for e in range(j + 1, len(b) + 1):
            subs_b.setdefault(b[j:e], []).append(j)
    for i in range(len(a)):
        for e in range(i + 1, len(a) + 1):
            w = a[i:e]
            if w in subs_b:
                if len(w) > best:
                    best, sa_, sb_ = len(w), set(), set()
                if len(w) == best:
                    sa_.add(i)
                    sb_.update(subs_b[w])
    return best, sorted(sa_), sorted(sb_)


def test_lcs_dp_against_substring_enumeration(oracle_mod):
    assert oracle_mod.lcs_dp(b"GATTACA", b"TTAC")[0] == 4
    assert oracle_mod.lcs_dp(b"AAAA", b"CCC")[0] == 0
    for seed in range(40):
        a, b = gen.fuzz_sequences(seed, nseq=2, max_len=25,
                                  alphabet=b"AC" if seed % 3 == 0 else b"ACGT")
        L, pa, pb = oracle_mod.lcs_dp(a, b)
        rL, rpa, rpb = _brute_lcs(bytes(a), bytes(b))
        assert L == rL
        if L:
            assert pa.tolist() == rpa and pb.tolist() == rpb


# ---------------------------------------------------------------- overlap pins

def _check_overlap_vs_dp(oracle_mod, seqs):
    text, starts, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text)
    lcp = oracle_mod.lcp_array(text, sa)
    ov = oracle_mod.longest_overlap(text, sa, lcp, starts)
    L, pos = oracle_mod.overlap_by_dp(seqs)
    assert ov["length"] == L
    assert ov["positions"].tolist() == pos.tolist()
    if L == 0:
        assert ov["rank"] == -1 and ov["seq_a"] == -1
        return ov
    # the canonical pair really shares L symbols and sits at adjacent ranks
    k = ov["rank"]
    assert lcp[k] == L and k >= 1
    pa = starts[ov["seq_a"]] + ov["pos_a"]
    pb = starts[ov["seq_b"]] + ov["pos_b"]
    assert ov["seq_a"] < ov["seq_b"]
    assert {int(pa), int(pb)} == {int(sa[k - 1]), int(sa[k])}
    assert np.array_equal(text[pa:pa + L], text[pb:pb + L])
    # smallest rank: no earlier cross pair reaches L
    sq = oracle_mod.seq_of(sa, starts)
    for kk in range(1, k):
        assert not (sq[kk] != sq[kk - 1] and lcp[kk] >= L)
    return ov


def test_overlap_fuzz_against_dp(oracle_mod):
    for seed in range(120):
        nseq = 2 if seed % 4 else 3
        alpha = [b"ACGT", b"AC", b"A"][seed % 3]
        seqs = gen.fuzz_sequences(1000 + seed, nseq=nseq, max_len=40, alphabet=alpha)
        _check_overlap_vs_dp(oracle_mod, seqs)


@pytest.mark.parametrize("name", sorted(gen.degenerate_cases()))
def test_overlap_degenerate_against_dp(oracle_mod, name):
    _check_overlap_vs_dp(oracle_mod, gen.degenerate_cases()[name])


def _assert_covers(ov, start, plant_len):
    """Some listed occurrence of the length-L region contains the plant (the
    plant may extend by chance when neighbouring bases agree)."""
    L = ov["length"]
    assert any(p <= start and start + plant_len <= p + L for p in ov["positions"].tolist())


def test_overlap_planted_pair_against_dp(oracle_mod):
    seqs, info = gen.pair_uniform(n_each=20_000, plant_len=500, seed=77)
    ov = _check_overlap_vs_dp(oracle_mod, seqs)
    assert ov["length"] >= 500
    o1, o2 = info["plant_offsets"]
    _assert_covers(ov, o1, 500)
    _assert_covers(ov, 20_001 + o2, 500)


def test_overlap_tiny_workload_planted_invariant(oracle_mod):
    seqs, info = gen.pair_uniform()            # 2 x 100,000, 500-base plant
    text, starts, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text, nthreads=4)
    assert oracle_mod.check_suffix_array(text, sa, nthreads=4) == -1
    lcp = oracle_mod.lcp_array(text, sa, nthreads=4)
    ov = oracle_mod.longest_overlap(text, sa, lcp, starts)
    assert ov["length"] >= 500
    o1, o2 = info["plant_offsets"]
    _assert_covers(ov, o1, 500)
    _assert_covers(ov, int(starts[1]) + o2, 500)


# ---------------------------------------------------------------- encoding

def test_encode_concat_codes_and_errors(oracle_mod):
    text, starts, sigma = oracle_mod.encode_concat([b"AC", b"gt"])
    assert text.tolist() == [3, 4, 2, 5, 6, 1]
    assert starts.tolist() == [0, 3, 6] and sigma == 7
    with pytest.raises(ValueError):
        oracle_mod.encode_concat([b"ACN", b"GT"])


# ---------------------------------------------------------------- int64 index variants

def test_int64_checks_against_python_string_order(oracle_mod):
    # brute force: Python's string order and os.path.commonprefix
    for s in ["GATTACA", "AAAAAA", "ACACAC", "TGCATGCA", "CAGTTGAC"]:
        text, _ = oracle_mod.encode_raw(s.encode())
        ref = sorted(range(len(s)), key=lambda i: s[i:])
        sa = np.array(ref, np.int64)
        assert oracle_mod.check_suffix_array64(text, sa) == -1
        ref_lcp = [0] + [len(os.path.commonprefix([s[ref[k - 1]:], s[ref[k]:]])) for k in range(1, len(s))]
        assert oracle_mod.lcp_array64(text, sa).tolist() == ref_lcp
        p = np.array([i for i in range(len(s)) for _ in range(len(s))], np.int64)
        q = np.array([j for _ in range(len(s)) for j in range(len(s))], np.int64)
        ref_q = [len(os.path.commonprefix([s[i:], s[j:]])) for i, j in zip(p.tolist(), q.tolist())]
        assert oracle_mod.lcp_pairs64(text, p, q).tolist() == ref_q


def test_int64_check_rejects_wrong_arrays(oracle_mod):
    seqs, _ = gen.pair_uniform(n_each=700, plant_len=40, seed=4)
    text, _, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text).astype(np.int64)
    assert oracle_mod.check_suffix_array64(text, sa, nthreads=3) == -1
    bad = sa.copy()
    bad[20], bad[21] = bad[21], bad[20]
    assert oracle_mod.check_suffix_array64(text, bad) == 21
    dup = sa.copy()
    dup[5] = dup[6]
    assert oracle_mod.check_suffix_array64(text, dup) == len(text)
    wide = sa.copy()
    wide[0] = 2**32 + int(sa[0])  # would alias sa[0] if truncated to 32 bits
    assert oracle_mod.check_suffix_array64(text, wide) == len(text)


def test_longest_overlap_large_against_dp(oracle_mod):
    # the scan-and-runs form gives the record and positions the DP fixes
    for seed in range(80):
        nseq = 2 if seed % 3 else 3
        alpha = [b"ACGT", b"AC", b"A", b"GT"][seed % 4]
        seqs = gen.fuzz_sequences(5000 + seed, nseq=nseq, max_len=40, alphabet=alpha)
        text, starts, _ = oracle_mod.encode_concat(seqs)
        sa = oracle_mod.suffix_array(text)
        lcp = oracle_mod.lcp_array(text, sa)
        got = oracle_mod.longest_overlap_large(text, sa.astype(np.int64), lcp, starts)
        exp = _check_overlap_vs_dp(oracle_mod, seqs)
        for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
            assert got[k] == exp[k], (seed, k)
        assert got["positions"].tolist() == exp["positions"].tolist(), seed


def test_overlap_max_scan_chunks_do_not_change_the_answer(oracle_mod):
    seqs, _ = gen.pair_noncoding(n_each=30_000, seed=9, shared_len=2000, core=400)
    text, starts, _ = oracle_mod.encode_concat(seqs)
    sa = oracle_mod.suffix_array(text, nthreads=4)
    lcp = oracle_mod.lcp_array(text, sa, nthreads=4)
    ov = oracle_mod.longest_overlap(text, sa, lcp, starts)
    for chunk in (1, 7, 4096, 1 << 24):
        assert oracle_mod.overlap_max_scan(sa, lcp, starts, chunk=chunk) == (ov["length"], ov["rank"])


# ---------------------------------------------------------------- many independent pairs

def test_pair_overlaps_against_the_dp_and_direct_comparison(oracle_mod):
    """The per-pair oracle of the batched and served workloads: each pair's
    length and position set equal the longest-common-substring DP's on that
    pair alone (Section 3 problem statement); each (p, q) answer equals the
    common prefix of the two suffixes of S1#S2$ counted by plain Python
    comparison; the records come back in pair order from the spawned worker
    pool (interleaved chunks put back in place) exactly as from one process."""
    rng = np.random.default_rng(31)
    pairs, queries = [], []
    for i in range(11):
        alpha = b"AC" if i % 4 == 0 else b"ACGT"
        la, lb = int(rng.integers(1, 90)), int(rng.integers(1, 90))
        a = np.frombuffer(alpha, np.uint8)[rng.integers(0, len(alpha), la)]
        b = np.frombuffer(alpha, np.uint8)[rng.integers(0, len(alpha), lb)]
        if i % 3 == 1 and la > 10:
            b = np.concatenate([b, a[3:3 + int(rng.integers(1, la - 3))]])  # a planted shared piece
        pairs.append((a, b))
        n = la + b.size + 2
        queries.append((rng.integers(0, n, 20).astype(np.int32), rng.integers(0, n, 20).astype(np.int32)))
    one = [oracle_mod.pair_overlap(a, b, q) for (a, b), q in zip(pairs, queries)]
    pooled = oracle_mod.pair_overlaps(pairs, queries=queries, processes=2)
    for (a, b), q, r, s in zip(pairs, queries, one, pooled):
        L, pos = oracle_mod.overlap_by_dp([a, b])
        assert r["length"] == L
        assert r["positions"].tolist() == pos.tolist()
        text = bytes(a) + b"#" + bytes(b) + b"$"  # the pair's text; separators are unique symbols
        for p_, q_, got in zip(q[0].tolist(), q[1].tolist(), r["answers"].tolist()):
            x, y, h = text[p_:], text[q_:], 0
            while h < min(len(x), len(y)) and x[h] == y[h]:
                h += 1
            assert got == h, (p_, q_)
        assert set(r) == set(s)
        for key in r:
            assert np.array_equal(np.asarray(r[key]), np.asarray(s[key])), key
