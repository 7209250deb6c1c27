"""Launch parameters change only speed: the whole path and the batched path
under every non-default value of every parameter, against the oracle, and
the autotuner's choice on a small batch."""
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
    yield lor
    lor.tune_set(**lor.tune_default())


@pytest.fixture(scope="module")
def O():
    import oracle
    oracle.build()
    return oracle


CONFIGS = [dict(digit_bits=6), dict(digit_bits=7), dict(level0_key_bits=30), dict(level0_key_bits=56),
           dict(sort_items_64=8), dict(sort_items_64=16), dict(sort_items_32=12), dict(merge_items=2), dict(merge_items=8),
           dict(digit_bits=5, level0_key_bits=24, sort_items_64=8, sort_items_32=12, merge_items=2)]


def expect_pair(O, a, b):
    text, starts, _ = O.encode_concat([a, b])
    sa = O.suffix_array(text)
    lcp = O.lcp_array(text, sa)
    return O.longest_overlap(text, sa, lcp, starts)


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: ",".join(f"{k}={v}" for k, v in c.items()))
def test_whole_path_and_batch_under_each_parameter(L, O, cfg):
    L.tune_set(**L.tune_default())
    L.tune_set(**cfg)
    try:
        seqs, _ = gen.pair_noncoding(n_each=60_000, seed=33, shared_len=3000, core=700)
        text, starts, sigma = O.encode_concat(seqs)
        ascii_dev = torch.from_numpy(np.concatenate(seqs)).cuda()
        t, st, _ = L.encode_concat(ascii_dev, [len(s) for s in seqs])
        sa = L.build_sa(t, sigma)
        isa, lcp = L.lcp(t, sa)
        L.check_device(where=str(cfg))
        sa_o = O.suffix_array(text)
        np.testing.assert_array_equal(sa.cpu().numpy(), sa_o)
        np.testing.assert_array_equal(lcp.cpu().numpy(), O.lcp_array(text, sa_o))
        pairs = gen.pair_batch(npairs=40, lo=500, hi=20_000, seed=140434492)
        flat = [s for pr in pairs for s in pr]
        b = L.lor.Batch([len(s) for s in flat])
        b.run(torch.from_numpy(np.concatenate(flat)).cuda())
        L.check_device(where=f"batch {cfg}")
        res = b.results()
        for p, (x, y) in enumerate(pairs):
            e = expect_pair(O, x, y)
            for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
                assert res[p][k] == e[k], (cfg, p, k)
            np.testing.assert_array_equal(res[p]["positions"], e["positions"])
    finally:
        L.tune_set(**L.tune_default())


def test_autotuner_picks_a_valid_configuration(L, O):
    L.tune_set(**L.tune_default())
    pairs = gen.pair_batch(npairs=64, lo=1_000, hi=30_000, seed=140434493)
    flat = [s for pr in pairs for s in pr]
    ascii_dev = torch.from_numpy(np.concatenate(flat)).cuda()
    b = L.lor.Batch([len(s) for s in flat])
    try:
        best, ms = L.autotune_batch(b, ascii_dev, reps=1)
        assert ms > 0
        assert L.tune_get() == best
        b.run(ascii_dev)
        L.check_device(where="after autotune")
        res = b.results()
        for p in range(0, len(pairs), 7):
            e = expect_pair(O, *pairs[p])
            assert res[p]["length"] == e["length"] and res[p]["rank"] == e["rank"]
            np.testing.assert_array_equal(res[p]["positions"], e["positions"])
    finally:
        L.tune_set(**L.tune_default())
