"""GPU path vs the CPU oracle, element by element, through the C ABI.

Every output of the path is an exact integer, so every comparison is
bit-exact: encoded text, suffix array, inverse suffix array, LCP array,
overlap record and its position list, sparse table and LCP-query answers.
Sizes span several kernel tiles with ragged tails; the full-size instances
(2 x 16,777,216 noncoding-like and 2 x 134,217,728 uniform bases) run in the
same configuration the benchmark times.
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


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.cuda() if dtype is None else t.to(dtype).cuda()


def gpu_path(L, seqs, queries=None, pos_cap=1 << 20, rmq=True):
    lens = [len(s) for s in seqs]
    ascii_dev = to_dev(np.concatenate(seqs) if sum(lens) else np.zeros(0, np.uint8))
    pipe = L.Pipeline(lens, pos_cap=pos_cap, with_rmq=rmq)
    p = q = ans = None
    if queries is not None:
        p, q = to_dev(queries[0]), to_dev(queries[1])
        ans = torch.empty_like(p)
    out, pos = pipe.run(ascii_dev, p, q, ans)
    L.check_device(where="gpu_path")
    res = dict(text=pipe.text.cpu().numpy(), starts=pipe.starts.cpu().numpy(),
               sa=pipe.sa.cpu().numpy(), isa=pipe.isa.cpu().numpy(), lcp=pipe.lcp.cpu().numpy(),
               overlap=L.overlap_dict(out, pos), n=pipe.n)
    if rmq:
        res["table"] = pipe.table
    if ans is not None:
        res["answers"] = ans.cpu().numpy()
    return res


def oracle_path(O, seqs, nthreads=1):
    text, starts, sigma = O.encode_concat(seqs)
    sa = O.suffix_array(text, nthreads=nthreads)
    lcp = O.lcp_array(text, sa, nthreads=nthreads)
    return dict(text=text, starts=starts, sa=sa, isa=O.inverse_suffix_array(sa), lcp=lcp,
                overlap=O.longest_overlap(text, sa, lcp, starts))


def assert_overlap_equal(got, exp):
    for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
        assert got[k] == exp[k], (k, got[k], exp[k])
    assert got["n_pos"] == len(exp["positions"])
    np.testing.assert_array_equal(got["positions"], exp["positions"])


def assert_full_parity(O, g, e, table=True):
    np.testing.assert_array_equal(g["text"], e["text"])
    np.testing.assert_array_equal(g["starts"], e["starts"].astype(np.int32))
    np.testing.assert_array_equal(g["sa"], e["sa"])
    np.testing.assert_array_equal(g["isa"], e["isa"])
    np.testing.assert_array_equal(g["lcp"], e["lcp"])
    assert_overlap_equal(g["overlap"], e["overlap"])
    if table and "table" in g:
        st = O.sparse_table(e["lcp"])
        from paper_1404_3448_gb300 import lor as C
        np.testing.assert_array_equal(C.table_view(g["table"], g["n"]).cpu().numpy(), st)


# ------------------------------------------------------------------ paper example

def test_paper_table1_raw_text(L, O):
    from golden.load import load
    g = load("paper_example.txt")
    codes = {"A": 1, "C": 2, "G": 3, "T": 4}
    text = np.array([codes[c] for c in g["text"][0]], dtype=np.uint8)
    t = to_dev(text)
    sa = L.build_sa(t, 5)
    isa, lcp = L.lcp(t, sa)
    L.check_device()
    assert sa.cpu().tolist() == g["sa"]
    assert (isa.cpu().numpy() + 1).tolist() == g["ranks1"]
    assert lcp.cpu().tolist() == g["lcp"]


# ------------------------------------------------------------------ encoding

def test_encode_matches_oracle(L, O):
    rng = np.random.default_rng(3)
    alpha = np.frombuffer(b"ACGTacgt", np.uint8)
    for nseq in [1, 2, 3, 17, 250]:
        seqs = [alpha[rng.integers(0, 8, int(rng.integers(0, 40)))] for _ in range(nseq)]
        lens = [len(s) for s in seqs]
        text, starts, sigma = L.encode_concat(to_dev(np.concatenate(seqs)), lens)
        L.check_device()
        et, es, esig = O.encode_concat(seqs)
        assert sigma == esig
        np.testing.assert_array_equal(text.cpu().numpy(), et)
        np.testing.assert_array_equal(starts.cpu().numpy(), es.astype(np.int32))


def test_encode_bad_symbol_reports_status(L):
    seqs = [np.frombuffer(b"ACGNT", np.uint8), np.frombuffer(b"GG", np.uint8)]
    L.encode_concat(to_dev(np.concatenate(seqs)), [5, 2])
    assert L.device_status() == -2
    assert L.device_status() == 0  # cleared


# ------------------------------------------------------------------ fuzz

# How DC3 orders each level: "auto" (the library's choice), "sort" (radix
# sort at every level and full recursion), "dbl" (prefix doubling of the
# reduced string whenever a sorted level's names repeat).
STRATEGIES = ["auto", "sort", "dbl"]


@pytest.fixture
def route(L):
    """Sets a DC3 route (lor_dc3_route_set) for one test, then the default."""
    def set_strategy(strategy="auto", k0=0):
        if strategy == "sort":
            L.dc3_route_set(k0, "sort", "never")
        elif strategy == "dbl":
            L.dc3_route_set(k0, "auto", "force")
        elif strategy == "sortdbl":
            L.dc3_route_set(k0, "sort", "force")
        elif strategy == "nodbl":
            L.dc3_route_set(k0, "auto", "never")
        else:
            L.dc3_route_set(k0)
    yield set_strategy
    L.dc3_route_set()



@pytest.mark.parametrize("strategy", STRATEGIES)
def test_fuzz_small_full_path(L, O, strategy, route):
    route(strategy)
    for seed in range(60):
        nseq = [2, 2, 3, 5][seed % 4]
        alpha = [b"ACGT", b"AC", b"A", b"ACGT"][seed % 4 if seed % 7 else 2]
        seqs = gen.fuzz_sequences(5000 + seed, nseq=nseq, max_len=[8, 40, 300][seed % 3],
                                  alphabet=alpha)
        e = oracle_path(O, seqs)
        rng = np.random.default_rng(seed)
        n = len(e["text"])
        p = rng.integers(0, n, 64).astype(np.int32)
        q = rng.integers(0, n, 64).astype(np.int32)
        g = gpu_path(L, seqs, (p, q))
        assert_full_parity(O, g, e)
        np.testing.assert_array_equal(g["answers"], O.lcp_pairs(e["text"], p, q))


@pytest.mark.parametrize("name", sorted(gen.degenerate_cases()))
def test_degenerate_inputs(L, O, name):
    seqs = gen.degenerate_cases()[name]
    e = oracle_path(O, seqs)
    n = len(e["text"])
    p, q = np.meshgrid(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32))
    g = gpu_path(L, seqs, (p.ravel().copy(), q.ravel().copy()))
    assert_full_parity(O, g, e)
    np.testing.assert_array_equal(g["answers"], O.lcp_pairs(e["text"], p.ravel(), q.ravel()))


# ------------------------------------------------------------------ tile spans

SIZES = [1, 2, 3, 4, 5, 6, 7, 31, 32, 33, 1023, 1024, 1025, 2047, 2048, 2049, 4095, 4096, 4097,
         6143, 6144, 8191, 8193, 12287, 65537, 131071, 300001]


@pytest.mark.parametrize("strategy", STRATEGIES)
@pytest.mark.parametrize("alpha", [b"ACGT", b"AC", b"A"])
def test_sizes_span_tiles(L, O, alpha, strategy, route):
    route(strategy)
    rng = np.random.default_rng(len(alpha))
    a = np.frombuffer(alpha, np.uint8)
    for total in SIZES:
        if alpha == b"A" and total > 13000:
            continue  # the oracle's comparison sort is quadratic on one-symbol runs
        l1 = int(rng.integers(0, total + 1))
        seqs = [a[rng.integers(0, a.size, l1)], a[rng.integers(0, a.size, total - l1)]]
        e = oracle_path(O, seqs, nthreads=NCPU)
        g = gpu_path(L, seqs, rmq=total < 5000)
        assert_full_parity(O, g, e, table=total < 5000)


@pytest.mark.parametrize("strategy", STRATEGIES + ["nodbl"])
@pytest.mark.parametrize("k0", ["3", "4", "7", "10", "21"])
def test_level0_prefix_lengths(L, O, k0, strategy, route):
    route(strategy, int(k0))
    seqs, _ = gen.pair_noncoding(n_each=150_000, seed=31, shared_len=4000, core=900)
    e = oracle_path(O, seqs, nthreads=NCPU)
    g = gpu_path(L, seqs, rmq=False)
    assert_full_parity(O, g, e, table=False)


def test_deep_recursion_single_symbol(L, O):
    # names stay few at every level, so no level is replaced by doubling
    seqs = [np.full(20000, ord("A"), np.uint8), np.full(15001, ord("A"), np.uint8)]
    e = oracle_path(O, seqs, nthreads=NCPU)
    g = gpu_path(L, seqs, rmq=False)
    assert_full_parity(O, g, e, table=False)
    trace = L.last_dc3_trace()
    last = trace[-1]
    assert len(trace) >= 8 and last["names"] == (last["n"] + 2) // 3 + last["n"] // 3
    assert "doubling" not in {t["strategy"] for t in trace}


@pytest.mark.parametrize("seqlen", [35001, 4096])
def test_doubling_on_one_symbol_runs(L, O, seqlen, route):
    # forced doubling from level 0: every group splits by one suffix per pass
    route("sortdbl")
    seqs = [np.full(seqlen, ord("A"), np.uint8), np.full(seqlen // 2, ord("A"), np.uint8)]
    e = oracle_path(O, seqs, nthreads=NCPU)
    g = gpu_path(L, seqs, rmq=False)
    assert_full_parity(O, g, e, table=False)
    trace = L.last_dc3_trace()
    assert [t["strategy"] for t in trace] == ["sort", "doubling"], trace


def test_wide_triples_two_stage_sort(L, O, route):
    # radix sorts at every level: level-2 names need > 21 bits, so level-3
    # triples exceed 64 bits
    route("sort", 3)
    seqs, _ = gen.pair_uniform(n_each=4_500_000, plant_len=700, seed=41)
    e = oracle_path(O, seqs, nthreads=NCPU)
    g = gpu_path(L, seqs, rmq=False)
    trace = L.last_dc3_trace()
    assert any(t["key_bits"] > 64 for t in trace), trace
    assert_full_parity(O, g, e, table=False)


# ------------------------------------------------------------------ level-0 key forms

def _raw_text_case(case, rng):
    """Raw code texts (no separators; the padding past the end is the only
    implicit smallest symbol) that reach the level-0 key forms, long enough
    (past 2^20 symbols) for the LCP's direct route."""
    if case == "dna_few_low_codes":
        # the four largest codes of sigma 21 plus a repeated motif holding the
        # low code 3 twice, so that several exception windows are equal
        t = rng.integers(17, 21, 1_200_000).astype(np.uint8)
        motif = np.array([18, 19, 3, 20, 17, 3, 3, 18, 18, 20, 17, 19, 20, 20, 17, 18, 19, 20], np.uint8)
        for pos in rng.choice(t.size - 64, 120, replace=False):
            t[pos:pos + motif.size] = motif
        t[rng.choice(t.size, 40, replace=False)] = rng.integers(1, 17, 40)
        return t, 21
    if case == "many_low_codes":  # exception windows everywhere: base-sigma keys
        return rng.integers(1, 21, 1_100_000).astype(np.uint8), 21
    if case == "two_codes":  # sigma 3: both codes take 2-bit values
        return rng.integers(1, 3, 1_100_000).astype(np.uint8), 3
    if case == "tail_run":  # a run of one symbol to the end: exception windows share keys
        t = rng.integers(1, 5, 1_100_000).astype(np.uint8)
        t[-300:] = 1
        return t, 5
    raise ValueError(case)


@pytest.mark.parametrize("case", ["dna_few_low_codes", "many_low_codes", "two_codes", "tail_run"])
@pytest.mark.parametrize("k0", [0, 1])
def test_level0_key_forms_on_raw_codes(L, O, case, k0, route):
    """Level 0's 2-bit keys (16 symbols, an exception bit, exception windows
    ordered by their symbols) and the base-sigma keys give the suffix array
    of the definition; a text with too many exception windows takes the
    base-sigma keys."""
    route("auto", k0)
    t, sigma = _raw_text_case(case, np.random.default_rng(sum(map(ord, case))))
    text = to_dev(t)
    sa = L.build_sa(text, sigma)
    L.check_device()
    sa_np = sa.cpu().numpy()
    np.testing.assert_array_equal(sa_np, O.suffix_array(t, nthreads=NCPU))
    if k0 == 0:  # the LCP of these texts: exceptions listed, or (many low codes) in the bitmap
        isa, lcp = L.lcp(text, sa)
        L.check_device()
        np.testing.assert_array_equal(lcp.cpu().numpy(), O.lcp_array(t, sa_np, nthreads=NCPU))
        np.testing.assert_array_equal(isa.cpu().numpy()[sa_np], np.arange(t.size, dtype=np.int32))
    two_bit = k0 == 0 and case != "many_low_codes"
    assert (L.last_dc3_trace()[0]["key_bits"] == 33) == two_bit, L.last_dc3_trace()


# ------------------------------------------------------------------ LCP routes

def _repeat_case(case, rng):
    """Two random sequences with one shared stretch: LCPs past 64 symbols at
    about 2 * length ranks, the longest about `length`."""
    length = {"no_repeat": 0, "repeat_5k": 5_000, "repeat_12k": 12_000, "repeat_many": 300_000}[case]
    a = rng.integers(0, 4, 1_200_000)
    b = rng.integers(0, 4, 1_000_000)
    if length:
        core = rng.integers(0, 4, length)
        a[100_000:100_000 + length] = core
        b[400_000:400_000 + length] = core
    alpha = np.frombuffer(b"ACGT", np.uint8)
    return [alpha[a], alpha[b]]


@pytest.mark.parametrize("case", ["no_repeat", "repeat_5k", "repeat_12k", "repeat_many"])
def test_lcp_direct_comparison_and_kasai_routes(L, O, case):
    """LCP in rank order by direct comparison (capped, with the long ranks
    finished separately) and, for a repeat past the comparison budget or too
    many long ranks, Kasai's method: both equal to the oracle's LCP by direct
    comparison, and ISA the inverse of SA."""
    seqs = _repeat_case(case, np.random.default_rng(sum(map(ord, case))))
    lens = [len(s) for s in seqs]
    text, _, sigma = L.encode_concat(to_dev(np.concatenate(seqs)), lens)
    sa = L.build_sa(text, sigma)
    isa, lcp = L.lcp(text, sa)
    L.check_device()
    t_np, sa_np = text.cpu().numpy(), sa.cpu().numpy()
    np.testing.assert_array_equal(lcp.cpu().numpy(), O.lcp_array(t_np, sa_np, nthreads=NCPU))
    np.testing.assert_array_equal(isa.cpu().numpy()[sa_np], np.arange(t_np.size, dtype=np.int32))


# ------------------------------------------------------------------ radix sort primitive

@pytest.mark.parametrize("m,bits,dups", [(0, 8, True), (1, 8, True), (4095, 12, True), (4097, 33, True),
                                         (100_003, 64, True), (300_000, 9, True),
                                         (200_000, 40, False), (70_001, 16, False)])
def test_radix_sort_primitive(L, O, m, bits, dups):
    """Stable sort against the paper's split sort (Section 4, Algorithm 1),
    with a third of the keys equal (one digit crowded in every pass) and with
    spread keys (equal low bits only by chance)."""
    rng = np.random.default_rng(m + bits)
    hi = (1 << min(bits + 2, 63)) - 1
    keys = rng.integers(0, hi, m, dtype=np.int64).astype(np.uint64)
    if dups and m > 10:
        keys[: m // 3] = keys[m // 3]  # heavy duplicates exercise stability
    vals = np.arange(m, dtype=np.uint32)[::-1].copy()
    k_t = to_dev(keys.view(np.int64))
    v_t = to_dev(vals.view(np.int32))
    if m:
        L.radix_sort_pairs(k_t, v_t, bits)
    L.check_device()
    ek, ev = O.radix_sort_split(keys, bits, values=vals.astype(np.int64))
    np.testing.assert_array_equal(k_t.cpu().numpy().view(np.uint64), ek)
    np.testing.assert_array_equal(v_t.cpu().numpy().view(np.uint32), ev.astype(np.uint32))


# ------------------------------------------------------------------ workloads

def test_tiny_workload_2x100k(L, O):
    seqs, info = gen.pair_uniform()
    e = oracle_path(O, seqs, nthreads=NCPU)
    p, q = gen.random_queries(len(e["text"]), count=200_000, seed=1)
    g = gpu_path(L, seqs, (p, q))
    assert_full_parity(O, g, e)
    np.testing.assert_array_equal(g["answers"], O.lcp_pairs(e["text"], p, q))
    assert g["overlap"]["length"] >= info["plant_len"]


@pytest.fixture(scope="module")
def noncoding_16M(O):
    seqs, info = gen.pair_noncoding()
    e = oracle_path(O, seqs, nthreads=NCPU)
    p, q = gen.random_queries(len(e["text"]), count=200_000, seed=2)
    return seqs, info, e, p, q, O.lcp_pairs(e["text"], p, q)


@pytest.mark.parametrize("strategy", ["auto", "nodbl", "k3nodbl"])
def test_noncoding_workload_2x16M(L, O, noncoding_16M, strategy, route):
    # k3nodbl: level 0 named by triples: a dense level, then sorted and parent levels
    route("nodbl" if strategy == "k3nodbl" else strategy, 3 if strategy == "k3nodbl" else 0)
    seqs, info, e, p, q, answers = noncoding_16M
    g = gpu_path(L, seqs, (p, q), rmq=True)
    assert_full_parity(O, g, e, table=False)
    np.testing.assert_array_equal(g["answers"], answers)
    assert g["overlap"]["length"] >= info["core"]
    used = [t["strategy"] for t in L.last_dc3_trace()]
    if strategy == "k3nodbl":
        assert set(used) == {"dense", "sort", "parent"}, L.last_dc3_trace()
    elif strategy == "nodbl":
        assert used[0] == "sort" and "parent" in used and "doubling" not in used, L.last_dc3_trace()
    else:
        assert used[-1] == "doubling" and "sort" in used, L.last_dc3_trace()


def test_large_workload_2x128M(L, O):
    """Full-size instance: the SA is checked against its definition at every
    rank, the LCP against direct comparison at every rank, the ISA as its
    inverse, the overlap by the oracle's scan over those verified arrays plus
    the planted region, and 1M queries by direct comparison."""
    seqs, info = gen.pair_large()
    text, starts, _ = O.encode_concat(seqs)
    p, q = gen.random_queries(len(text), count=1_000_000)
    g = gpu_path(L, seqs, (p, q), pos_cap=1 << 16, rmq=True)
    assert L.last_dc3_trace()[-1]["strategy"] == "doubling", L.last_dc3_trace()
    del g["table"]
    np.testing.assert_array_equal(g["text"], text)
    assert O.check_suffix_array(text, g["sa"], nthreads=NCPU) == -1
    np.testing.assert_array_equal(g["lcp"], O.lcp_array(text, g["sa"], nthreads=NCPU))
    np.testing.assert_array_equal(g["isa"][g["sa"]], np.arange(len(text), dtype=np.int32))
    exp = O.longest_overlap(text, g["sa"], g["lcp"], starts)
    assert_overlap_equal(g["overlap"], exp)
    o1, o2 = info["plant_offsets"]
    Lr = exp["length"]
    assert Lr >= info["plant_len"]
    pos = exp["positions"].tolist()
    for start in (o1, int(starts[1]) + o2):
        assert any(x <= start and start + info["plant_len"] <= x + Lr for x in pos)
    np.testing.assert_array_equal(g["answers"], O.lcp_pairs(text, p, q))


# ------------------------------------------------------------------ device-side errors

def test_device_errors_are_reported_not_faulted(L):
    n = 1000
    text = to_dev(np.full(n, 5, np.uint8))
    bad_sa = to_dev(np.arange(n, dtype=np.int32))
    bad_sa[7] = n + 5
    isa = torch.empty(n, dtype=torch.int32, device="cuda")
    lcp = torch.empty(n, dtype=torch.int32, device="cuda")
    L.lcp(text, bad_sa, isa, lcp)
    assert L.device_status() == -7
    # out-of-range query positions give -1 and a status
    good_sa = L.build_sa(text, 7)
    isa, lcp = L.lcp(text, good_sa)
    table = L.rmq_build(lcp)
    p = to_dev(np.array([0, -1, n], np.int32))
    q = to_dev(np.array([1, 0, 0], np.int32))
    ans = L.rmq_query(table, isa, p, q)
    assert L.device_status() == -7
    assert ans.cpu().tolist()[1:] == [-1, -1]
    # a text code outside [1, sigma)
    bad_text = to_dev(np.array([5, 6, 0, 5, 9, 1], np.uint8))
    L.build_sa(bad_text, 7)
    assert L.device_status() == -2
    assert L.device_status() == 0
