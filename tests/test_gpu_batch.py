"""lor_batch_overlap against the oracle, pair by pair.

Every pair's record and position list must equal what the oracle computes for
that pair alone (its own text S1#S2$): batching is an implementation detail
that changes no result.  Batches here span several groups (up to 512 pairs
each), hold empty sequences, degenerate pairs and uneven lengths.
"""
import numpy as np
import pytest

import lor_inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3448_gb300 as lor
    lor.load()
    return lor


def run_batch(L, pairs, pos_cap=1 << 22):
    flat = [s for pr in pairs for s in pr]
    lens = [len(s) for s in flat]
    ascii_dev = torch.from_numpy(np.concatenate(flat) if sum(lens) else np.zeros(0, np.uint8)).cuda()
    b = L.lor.Batch(lens, pos_cap=pos_cap)
    b.run(ascii_dev)
    L.check_device(where="batch")
    return b.results()


def expect_pair(O, a, b):
    text, starts, _ = O.encode_concat([a, b])
    sa = O.suffix_array(text)
    lcp = O.lcp_array(text, sa)
    return O.longest_overlap(text, sa, lcp, starts)


def assert_same(got, exp, p):
    for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
        assert got[k] == exp[k], (p, k, got[k], exp[k])
    assert got["n_pos"] == len(exp["positions"]), p
    np.testing.assert_array_equal(got["positions"], exp["positions"], err_msg=str(p))


def test_batch_small_random_pairs_over_three_groups(L, oracle_mod):
    pairs = []
    for i in range(1100):
        alpha = [b"ACGT", b"AC", b"A"][i % 3]
        a, b = gen.fuzz_sequences(7000 + i, nseq=2, max_len=[5, 60, 400][i % 3], alphabet=alpha)
        if i % 17 == 0:
            a = a[:0]  # empty first sequence
        if i % 23 == 0:
            b = b[:0]
        pairs.append([a, b])
    res = run_batch(L, pairs)
    assert len(res) == len(pairs)
    for p, (a, b) in enumerate(pairs):
        assert_same(res[p], expect_pair(oracle_mod, a, b), p)


def test_batch_degenerate_pairs(L, oracle_mod):
    cases = [v for v in gen.degenerate_cases().values() if len(v) == 2]
    res = run_batch(L, cases)
    for p, (a, b) in enumerate(cases):
        assert_same(res[p], expect_pair(oracle_mod, a, b), p)


def test_batch_noncoding_pairs_of_uneven_length(L, oracle_mod):
    pairs = gen.pair_batch(npairs=160, lo=1_000, hi=60_000, seed=140434490)
    res = run_batch(L, pairs)
    for p, (a, b) in enumerate(pairs):
        assert_same(res[p], expect_pair(oracle_mod, a, b), p)


def test_batch_single_pair_equals_plain_path(L, oracle_mod):
    seqs, _ = gen.pair_uniform(n_each=50_000, plant_len=300, seed=5)
    res = run_batch(L, [seqs])
    assert_same(res[0], expect_pair(oracle_mod, *seqs), 0)


def test_batch_positions_capacity(L, oracle_mod):
    pairs = [[np.frombuffer(b"A" * 10, np.uint8), np.frombuffer(b"CAC", np.uint8)]] * 3
    res = run_batch(L, pairs, pos_cap=5)
    exp = expect_pair(oracle_mod, *pairs[0])
    assert res[0]["n_pos"] == len(exp["positions"])
    np.testing.assert_array_equal(res[0]["positions"], exp["positions"][:5])


def test_batch_repeated_pair_many_copies(L, oracle_mod):
    """300 copies of one pair in one group: the group text is one long
    repeat (pair texts share their terminator codes), yet every block must
    still be the pair's own suffix array."""
    seqs, _ = gen.pair_uniform(n_each=1500, plant_len=120, seed=77)
    pairs = [seqs] * 300 + [[seqs[1], seqs[0]]]
    res = run_batch(L, pairs)
    exp = expect_pair(oracle_mod, *seqs)
    for p in range(300):
        assert_same(res[p], exp, p)
    assert_same(res[300], expect_pair(oracle_mod, seqs[1], seqs[0]), 300)


# ------------------------------------------------------------------ CUDA graph replay

def graph_results(L, pairs, ascii_dev=None, pos_cap=1 << 22):
    flat = [s for pr in pairs for s in pr]
    lens = [len(s) for s in flat]
    if ascii_dev is None:
        ascii_dev = torch.from_numpy(np.concatenate(flat) if sum(lens) else np.zeros(1, np.uint8)).cuda()
    g = L.lor.BatchGraph(lens, ascii_dev, pos_cap=pos_cap)
    return g, ascii_dev


def test_batch_graph_replays_equal_eager_and_oracle(L, oracle_mod):
    """The captured pipeline (no host round trip; doubling rounds enqueued up
    front) gives every pair's record and positions, on two replays in a row,
    and again after the input bytes change under the same lengths."""
    pairs = []
    for i in range(700):  # two groups (at most 512 pairs each)
        alpha = [b"ACGT", b"AC", b"A"][i % 3]
        a, b = gen.fuzz_sequences(9100 + i, nseq=2, max_len=[5, 60, 300][i % 3], alphabet=alpha)
        if i % 19 == 0:
            a = a[:0]
        pairs.append([a, b])
    pairs += gen.pair_batch(npairs=12, lo=1_000, hi=40_000, seed=140434491)
    g, ascii_dev = graph_results(L, pairs)
    assert g.kernels > 0
    for rep in range(2):
        g.run()
        L.check_device(where=f"graph replay {rep}")
        res = g.results()
        for p, (a, b) in enumerate(pairs):
            assert_same(res[p], expect_pair(oracle_mod, a, b), (rep, p))
    # new bases, same lengths: the graph reads its input buffer at every replay
    rng = np.random.default_rng(5)
    alpha = np.frombuffer(b"ACGT", np.uint8)
    pairs2 = [[alpha[rng.integers(0, 4, len(a))], alpha[rng.integers(0, 4, len(b))]] for a, b in pairs]
    flat2 = np.concatenate([s for pr in pairs2 for s in pr])
    ascii_dev.copy_(torch.from_numpy(flat2))
    g.run()
    L.check_device(where="graph replay, new input")
    res = g.results()
    eager = run_batch(L, pairs2)
    for p, (a, b) in enumerate(pairs2):
        assert_same(res[p], {**eager[p], "positions": eager[p]["positions"]}, p)
        if p % 50 == 0:
            assert_same(res[p], expect_pair(oracle_mod, a, b), p)
    g.close()


def test_batch_graph_long_repeats(L, oracle_mod):
    """Copies of one pair make the group text one long repeat: many doubling
    rounds run inside the graph before every sample is resolved."""
    seqs, _ = gen.pair_uniform(n_each=1500, plant_len=120, seed=78)
    pairs = [seqs] * 200 + [[np.frombuffer(b"A" * 3000, np.uint8), np.frombuffer(b"A" * 700, np.uint8)]]
    g, _ = graph_results(L, pairs)
    g.run()
    L.check_device(where="graph replay, repeats")
    res = g.results()
    exp = expect_pair(oracle_mod, *seqs)
    for p in range(200):
        assert_same(res[p], exp, p)
    assert_same(res[200], expect_pair(oracle_mod, *pairs[200]), 200)
    g.close()


# ------------------------------------------------------------------ the full batched workload

@pytest.fixture(scope="module")
def batch4096(oracle_mod):
    """The batched workload at its stated size: 4096 noncoding-like pairs with
    per-sequence lengths log-uniform in [1k, 1M] (about 1.18e9 bases), and the
    oracle's record for every pair alone, computed on all host cores."""
    pairs = gen.pair_batch()
    return pairs, oracle_mod.pair_overlaps(pairs)


def _groups(pairs, cap_pairs=512, cap_symbols=1 << 28):
    """Pair ranges [p0, p1) of the groups lor_batch_overlap forms (consecutive
    pairs up to 512 pairs or 2^28 text symbols), to point at their edges."""
    out, p0, n = [], 0, 0
    for p, (a, b) in enumerate(pairs):
        add = len(a) + len(b) + 2
        if p > p0 and (p - p0 == cap_pairs or n + add > cap_symbols):
            out.append((p0, p))
            p0, n = p, 0
        n += add
    out.append((p0, len(pairs)))
    return out


def test_batch_4096_pairs_every_record_equals_oracle(L, batch4096):
    """Every pair of the full batched workload, eager and as one CUDA graph
    replayed twice: record and position list equal to the oracle's for that
    pair alone.  The batch spans eight 512-pair groups, so group edges, the
    pair-split pass over 2^27-symbol group texts and the segmented Kasai and
    overlap all run at size."""
    pairs, exp = batch4096
    groups = _groups(pairs)
    assert len(groups) >= 8 and max(p1 - p0 for p0, p1 in groups) == 512
    longest = max(range(len(pairs)), key=lambda p: len(pairs[p][0]) + len(pairs[p][1]))
    assert len(pairs[longest][0]) + len(pairs[longest][1]) > 1_500_000
    flat = [s for pr in pairs for s in pr]
    lens = [len(s) for s in flat]
    ascii_dev = torch.from_numpy(np.concatenate(flat)).cuda()
    pos_cap = 1 << 24
    b = L.lor.Batch(lens, pos_cap=pos_cap)
    b.run(ascii_dev)
    L.check_device(where="batch of 4096 pairs")
    res = b.results()
    for p in range(len(pairs)):
        assert_same(res[p], exp[p], p)
    del b
    g = L.lor.BatchGraph(lens, ascii_dev, pos_cap=pos_cap)
    for rep in range(2):
        g.run()
        L.check_device(where=f"graph of 4096 pairs, replay {rep}")
        res = g.results()
        for p in range(len(pairs)):
            assert_same(res[p], exp[p], (rep, p))
    g.close()
