"""The 64-bit index path (lor_*64) against the CPU oracle, through the C ABI.

Small and tile-spanning texts are compared element by element with the
oracle (suffix array, inverse suffix array, LCP array, overlap record and
positions, block-RMQ answers); the instance past 2^31 symbols is checked
against the definitions at every rank (suffix order, permutation, LCP by
direct comparison), the overlap by the oracle's scan over those verified
arrays plus the planted region past 2^31, and 1M queries by direct
comparison.
"""
import os

import numpy as np
import pytest

import lor_inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
NCPU = os.cpu_count() or 4


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3448_gb300 as lor
    lor.load()
    return lor


@pytest.fixture(scope="module")
def O(oracle_mod):
    return oracle_mod


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def path64(L, seqs, queries=None, pos_cap=1 << 20):
    lens = [len(s) for s in seqs]
    ascii_dev = to_dev(np.concatenate(seqs) if sum(lens) else np.zeros(0, np.uint8))
    text, starts, sigma = L.encode_concat64(ascii_dev, lens)
    del ascii_dev
    sa = L.build_sa64(text, sigma)
    isa, lcp = L.lcp64(text, sa)
    out, pos = L.longest_overlap64(sa, lcp, starts, len(seqs), pos_cap=pos_cap)
    res = dict(overlap=L.overlap64_dict(out, pos))
    if queries is not None:
        table = L.rmq_block_build(lcp)
        p, q = to_dev(queries[0]), to_dev(queries[1])
        res["answers"] = L.rmq_block_query64(table, lcp, isa, p, q).cpu().numpy()
        del table, p, q
    L.check_device(where="path64")
    res.update(text=text.cpu().numpy(), starts=starts.cpu().numpy(), sa=sa.cpu().numpy(),
               isa=isa.cpu().numpy(), lcp=lcp.cpu().numpy())
    return res


def oracle_path(O, seqs):
    text, starts, sigma = O.encode_concat(seqs)
    sa = O.suffix_array(text, nthreads=NCPU)
    lcp = O.lcp_array(text, sa, nthreads=NCPU)
    return dict(text=text, starts=starts, sa=sa, isa=O.inverse_suffix_array(sa), lcp=lcp,
                overlap=O.longest_overlap(text, sa, lcp, starts))


def assert_parity(g, e):
    np.testing.assert_array_equal(g["text"], e["text"])
    np.testing.assert_array_equal(g["starts"], e["starts"])
    assert g["sa"].dtype == np.int64 and g["isa"].dtype == np.int64
    np.testing.assert_array_equal(g["sa"], e["sa"])
    np.testing.assert_array_equal(g["isa"], e["isa"])
    np.testing.assert_array_equal(g["lcp"], e["lcp"])
    go, eo = g["overlap"], e["overlap"]
    for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
        assert go[k] == eo[k], (k, go[k], eo[k])
    assert go["n_pos"] == len(eo["positions"])
    np.testing.assert_array_equal(go["positions"], eo["positions"])


def test_paper_table1_raw_text(L, O):
    from golden.load import load
    g = load("paper_example.txt")
    codes = {"A": 1, "C": 2, "G": 3, "T": 4}
    text = to_dev(np.array([codes[c] for c in g["text"][0]], dtype=np.uint8))
    sa = L.build_sa64(text, 5)
    isa, lcp = L.lcp64(text, sa)
    L.check_device()
    assert sa.cpu().tolist() == g["sa"]
    assert (isa.cpu().numpy() + 1).tolist() == g["ranks1"]
    assert lcp.cpu().tolist() == g["lcp"]


def test_encode64_matches_oracle(L, O):
    rng = np.random.default_rng(11)
    alpha = np.frombuffer(b"ACGTacgt", np.uint8)
    for nseq in [1, 2, 5, 250]:
        seqs = [alpha[rng.integers(0, 8, int(rng.integers(0, 30)))] for _ in range(nseq)]
        text, starts, sigma = L.encode_concat64(to_dev(np.concatenate(seqs)), [len(s) for s in seqs])
        L.check_device()
        et, es, esig = O.encode_concat(seqs)
        assert sigma == esig and starts.dtype == torch.int64
        np.testing.assert_array_equal(text.cpu().numpy(), et)
        np.testing.assert_array_equal(starts.cpu().numpy(), es)


@pytest.mark.parametrize("name", sorted(gen.degenerate_cases()))
def test_degenerate_inputs(L, O, name):
    seqs = gen.degenerate_cases()[name]
    e = oracle_path(O, seqs)
    n = len(e["text"])
    p, q = np.meshgrid(np.arange(n, dtype=np.int64), np.arange(n, dtype=np.int64))
    g = path64(L, seqs, (p.ravel().copy(), q.ravel().copy()))
    assert_parity(g, e)
    np.testing.assert_array_equal(g["answers"], O.lcp_pairs64(e["text"], p.ravel(), q.ravel()))


def test_fuzz_small(L, O):
    rng = np.random.default_rng(64)
    for it in range(40):
        nseq = int(rng.integers(1, 6))
        alpha = np.frombuffer([b"ACGT", b"AC", b"A", b"GT"][it % 4], np.uint8)
        seqs = [alpha[rng.integers(0, alpha.size, int(rng.integers(0, 200)))] for _ in range(nseq)]
        e = oracle_path(O, seqs)
        n = len(e["text"])
        p = rng.integers(0, n, 64)
        q = rng.integers(0, n, 64)
        g = path64(L, seqs, (p, q))
        assert_parity(g, e)
        np.testing.assert_array_equal(g["answers"], O.lcp_pairs64(e["text"], p, q))


SIZES = [1, 2, 7, 31, 33, 2047, 2049, 4095, 4097, 8193, 65537, 300001]


@pytest.mark.parametrize("alpha", [b"ACGT", b"AC", b"A"])
def test_sizes_span_tiles(L, O, alpha):
    rng = np.random.default_rng(len(alpha) + 64)
    a = np.frombuffer(alpha, np.uint8)
    for total in SIZES:
        if alpha == b"A" and total > 13000:
            continue  # the oracle's comparison sort is quadratic on one-symbol runs
        l1 = int(rng.integers(0, total + 1))
        seqs = [a[rng.integers(0, a.size, l1)], a[rng.integers(0, a.size, total - l1)]]
        assert_parity(path64(L, seqs), oracle_path(O, seqs))


def test_one_symbol_runs_double_every_round(L, O):
    # every suffix ties with its neighbours until the doubled prefix covers it
    seqs = [np.full(35001, ord("A"), np.uint8), np.full(17500, ord("A"), np.uint8)]
    assert_parity(path64(L, seqs), oracle_path(O, seqs))


def test_noncoding_repeats(L, O):
    seqs, info = gen.pair_noncoding(n_each=150_000, seed=31, shared_len=4000, core=900)
    e = oracle_path(O, seqs)
    g = path64(L, seqs)
    assert_parity(g, e)
    assert g["overlap"]["length"] >= info["core"]


def test_int32_and_int64_paths_agree(L):
    seqs, _ = gen.pair_noncoding(n_each=1 << 20, seed=5, shared_len=4000, core=900)
    lens = [len(s) for s in seqs]
    ascii_dev = to_dev(np.concatenate(seqs))
    t32, st32, sigma = L.encode_concat(ascii_dev, lens)
    sa32 = L.build_sa(t32, sigma)
    isa32, lcp32 = L.lcp(t32, sa32)
    g = path64(L, seqs)
    np.testing.assert_array_equal(g["sa"], sa32.cpu().numpy())
    np.testing.assert_array_equal(g["isa"], isa32.cpu().numpy())
    np.testing.assert_array_equal(g["lcp"], lcp32.cpu().numpy())


def test_device_errors_are_reported(L):
    n = 1000
    text = to_dev(np.full(n, 5, np.uint8))
    bad = torch.arange(n, dtype=torch.int64, device="cuda")
    bad[7] = n + 5
    L.lcp64(text, bad)
    assert L.device_status() == L.lor.LOR_ERR_BAD_INPUT
    assert L.device_status() == 0
    text[3] = 9
    L.build_sa64(text, 6)
    assert L.device_status() == L.lor.LOR_ERR_BAD_SYMBOL
    assert L.device_status() == 0


def test_past_int32_range(L, O):
    """2 x (2^30 + 2^15) uniform bases, n = 2^31 + 2^16 + 2."""
    seqs, info = gen.pair_int64()
    lens = [len(s) for s in seqs]
    n = sum(lens) + 2
    assert n > 2**31
    p, q = gen.random_queries64(n, count=1_000_000)
    p[:4] = [n - 1, n - 2, 2**31 + 5, 0]
    q[:4] = [n - 1, 2**31 + 7, 2**31 + 5, n - 3]
    ascii_dev = to_dev(np.concatenate(seqs))
    text, starts, sigma = L.encode_concat64(ascii_dev, lens)
    del ascii_dev
    sa = L.build_sa64(text, sigma)
    torch.cuda.empty_cache()
    isa, lcp = L.lcp64(text, sa)
    torch.cuda.empty_cache()
    assert torch.equal(isa[sa], torch.arange(n, dtype=torch.int64, device="cuda"))
    out, pos = L.longest_overlap64(sa, lcp, starts, 2, pos_cap=1 << 16)
    table = L.rmq_block_build(lcp)
    ans = L.rmq_block_query64(table, lcp, isa, to_dev(p), to_dev(q))
    L.check_device(where="past_int32_range")
    got = L.overlap64_dict(out, pos)
    ans = ans.cpu().numpy()
    del table, isa, out, pos
    h_text = text.cpu().numpy()
    h_starts = starts.cpu().numpy()
    h_sa = sa.cpu().numpy()
    del sa
    h_lcp = lcp.cpu().numpy()
    del lcp, text
    torch.cuda.empty_cache()
    et, es, _ = O.encode_concat(seqs)
    np.testing.assert_array_equal(h_text, et)
    np.testing.assert_array_equal(h_starts, es)
    del et
    assert O.check_suffix_array64(h_text, h_sa, nthreads=NCPU) == -1
    np.testing.assert_array_equal(h_lcp, O.lcp_array64(h_text, h_sa, nthreads=NCPU))
    exp = O.longest_overlap_large(h_text, h_sa, h_lcp, h_starts)
    for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
        assert got[k] == exp[k], (k, got[k], exp[k])
    assert got["n_pos"] == len(exp["positions"])
    np.testing.assert_array_equal(got["positions"], exp["positions"])
    o1, o2 = info["plant_offsets"]
    assert exp["length"] >= info["plant_len"]
    far = int(h_starts[1]) + o2
    assert far > 2**31
    assert any(x <= far and far + info["plant_len"] <= x + exp["length"] for x in exp["positions"].tolist())
    np.testing.assert_array_equal(ans, O.lcp_pairs64(h_text, p, q))
