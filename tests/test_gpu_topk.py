"""The K longest left-maximal overlaps (lor_topk_overlaps) against the
oracle, entry by entry."""
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


def check(L, O, seqs, Ks):
    text, starts, sigma = O.encode_concat(seqs)
    t = torch.from_numpy(text).cuda()
    st = torch.from_numpy(np.asarray(starts, np.int32)).cuda()
    sa = L.build_sa(t, sigma)
    isa, lcp = L.lcp(t, sa)
    sa_o = O.suffix_array(text, nthreads=4)
    lcp_o = O.lcp_array(text, sa_o)
    for K in Ks:
        got = L.topk_overlaps(t, sa, lcp, st, len(seqs), K)
        L.check_device(where=f"topk K={K}")
        exp = O.topk_overlaps(text, sa_o, lcp_o, starts, K)
        assert len(got) == len(exp), (K, len(got), len(exp))
        for g, e in zip(got, exp):
            assert {k: g[k] for k in e} == e, (K, g, e)


def test_topk_small_and_degenerate(L, oracle_mod):
    rng = np.random.default_rng(31)
    A = np.frombuffer(b"ACGT", np.uint8)
    for trial in range(12):
        alpha = [A, A[:2], A[:1]][trial % 3]
        seqs = [alpha[rng.integers(0, alpha.size, int(rng.integers(1, 400)))] for _ in range(2 + trial % 4)]
        check(L, oracle_mod, seqs, [1, 7, 100])


def test_topk_noncoding_pair(L, oracle_mod):
    seqs, _ = gen.pair_noncoding(n_each=100_000, seed=35, shared_len=3000, core=600)
    check(L, oracle_mod, seqs, [1, 64, 4096])
