"""Host-only checks that the seeded input generators make the workloads they
are said to make: sizes, alphabet, the planted shared pieces at their recorded
offsets, the noncoding background's base mix, log-uniform lengths, Poisson
arrivals and in-range follow-up queries.  The generators draw random numbers
only; none of the method's arithmetic is involved."""
import numpy as np

import lor_inputs as gen

ACGT = set(b"ACGT")


def _is_dna(s):
    return s.dtype == np.uint8 and set(np.unique(s).tolist()) <= ACGT


def test_seeded_and_repeatable():
    a, ia = gen.pair_uniform(n_each=5000, plant_len=100, seed=7)
    b, ib = gen.pair_uniform(n_each=5000, plant_len=100, seed=7)
    c, _ = gen.pair_uniform(n_each=5000, plant_len=100, seed=8)
    assert all(np.array_equal(x, y) for x, y in zip(a, b)) and ia == ib
    assert not np.array_equal(a[0], c[0])


def test_pair_uniform_sizes_mix_and_plant():
    (s1, s2), info = gen.pair_uniform(n_each=200_000, plant_len=500, seed=gen.SEED_BASE + 1)
    assert s1.size == s2.size == 200_000 and _is_dna(s1) and _is_dna(s2)
    for s in (s1, s2):  # iid uniform: each base about a quarter
        frac = np.bincount(np.searchsorted(np.frombuffer(b"ACGT", np.uint8), s), minlength=4) / s.size
        assert np.all(np.abs(frac - 0.25) < 0.01)
    o1, o2 = info["plant_offsets"]
    assert np.array_equal(s1[o1:o1 + 500], s2[o2:o2 + 500])
    # the large workload is the same generator at 134,217,728 bases a sequence
    assert gen.SIZE_LARGE == 134_217_728
    (l1, _), linfo = gen.pair_large(n_each=3000)
    assert l1.size == 3000 and linfo["plant_len"] == 500


def test_pair_noncoding_background_repeats_and_shared_core():
    (s1, s2), info = gen.pair_noncoding(n_each=400_000)
    assert s1.size == s2.size == 400_000 and _is_dna(s1) and _is_dna(s2)
    for s in (s1, s2):  # 40 % GC background; repeats and microsatellites move it little
        gc = np.isin(s, np.frombuffer(b"CG", np.uint8)).mean()
        assert 0.37 < gc < 0.43
    o1, o2 = info["shared_offsets"]
    L, core = info["shared_len"], info["core"]
    c0 = (L - core) // 2
    assert np.array_equal(s1[o1 + c0:o1 + c0 + core], s2[o2 + c0:o2 + c0 + core])
    # outside the core the two copies differ at about 2 % of positions (1 % substitutions each)
    diff = np.mean(s1[o1:o1 + c0] != s2[o2:o2 + c0])
    assert 0.003 < diff < 0.05


def test_pair_batch_lengths_are_log_uniform():
    lo, hi = 1_000, 30_000
    pairs = gen.pair_batch(npairs=300, lo=lo, hi=hi, seed=3)
    lens = np.array([len(s) for p in pairs for s in p], dtype=np.float64)
    assert lens.min() >= lo and lens.max() <= hi
    assert all(_is_dna(s) for p in pairs[:20] for s in p)
    # log-uniform: the logs are uniform on [log lo, log hi] (mean and spread)
    u = (np.log(lens) - np.log(lo)) / (np.log(hi) - np.log(lo))
    assert abs(u.mean() - 0.5) < 0.04
    assert abs(u.std() - np.sqrt(1 / 12)) < 0.03


def test_poisson_arrivals_rate_and_order():
    t = gen.poisson_arrivals(2000, 5.0, seed=11)
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < 5.0
    assert abs(t.size - 10_000) < 4 * 100  # mean 10,000, standard deviation 100
    assert abs(np.diff(t).mean() - 1 / 2000) < 0.05 / 2000


def test_request_stream_queries_stay_inside_their_pair():
    lens = [(10, 20), (1000, 5), (7, 7)]
    choice, P, Q = gen.request_stream(500, lens, queries=16, seed=2)
    n = np.array([a + b + 2 for a, b in lens])[choice]
    assert P.shape == Q.shape == (500, 16)
    assert np.all(P >= 0) and np.all(Q >= 0)
    assert np.all(P < n[:, None]) and np.all(Q < n[:, None])
    assert set(choice.tolist()) == {0, 1, 2}


def test_multi_query_lengths_and_reads():
    ref, qs = gen.multi_query(ref_len=60_000, nq=120, lo=100, hi=2_000, seed=5)
    assert ref.size == 60_000 and _is_dna(ref)
    assert len(qs) == 120 and all(100 <= q.size <= 2_000 and _is_dna(q) for q in qs)
    # every second query is a read of the reference with 1-5 % substitutions:
    # some window of the reference matches it at 90 % of positions or more
    refb = ref.tobytes()
    for q in qs[:10:2]:
        k = 12  # an exact 12-mer of the read locates its window
        hits = [i for i in range(0, q.size - k, k) if refb.find(q[i:i + k].tobytes()) >= 0]
        assert hits, "no exact 12-mer of the read occurs in the reference"
        i = hits[0]
        off = refb.find(q[i:i + k].tobytes()) - i
        if 0 <= off <= ref.size - q.size:
            assert np.mean(ref[off:off + q.size] == q) >= 0.9


def test_pair_int64_plant_lies_near_the_end_of_the_second_sequence():
    (s1, s2), info = gen.pair_int64(n_each=20_000)
    o1, o2 = info["plant_offsets"]
    assert o2 == 20_000 - 500 - 100
    assert np.array_equal(s1[o1:o1 + 500], s2[o2:o2 + 500])
    # at full size the copy's text position (after S1 and its terminator) passes 2^31
    assert gen.SIZE_INT64 + 1 + (gen.SIZE_INT64 - 600) > 2 ** 31
