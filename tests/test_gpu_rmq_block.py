"""Linear-space (block-sparse) RMQ against the oracle: the table of block
minima windows element by element, and LCP queries between arbitrary
suffixes against direct comparison, at sizes around the 32-entry block and
on a 2 x 1,000,000-base instance."""
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


def block_view(C, table, n):
    nb = -(-n // 32)
    stride = (nb + 63) // 64 * 64
    levels = max(1, nb.bit_length())
    return table[: levels * stride].view(levels, stride)[:, :nb]


def run_case(L, O, seqs, nq, seed, all_pairs=False):
    from paper_1404_3448_gb300 import lor as C
    text, starts, sigma = O.encode_concat(seqs)
    n = text.size
    t = torch.from_numpy(text).cuda()
    sa = L.build_sa(t, sigma)
    isa, lcp = L.lcp(t, sa)
    table = L.rmq_block_build(lcp)
    if all_pairs:
        pp, qq = np.meshgrid(np.arange(n, dtype=np.int32), np.arange(n, dtype=np.int32))
        p, q = pp.ravel().copy(), qq.ravel().copy()
    else:
        p, q = gen.random_queries(n, count=nq, seed=seed)
    pd, qd = torch.from_numpy(p).cuda(), torch.from_numpy(q).cuda()
    ans = L.rmq_block_query(table, lcp, isa, pd, qd)
    val, arg = L.rmq_block_argmin(table, lcp, isa, pd, qd)
    L.check_device(where="block rmq")
    sa_o = O.suffix_array(text)
    lcp_o = O.lcp_array(text, sa_o)
    np.testing.assert_array_equal(lcp.cpu().numpy(), lcp_o)
    np.testing.assert_array_equal(block_view(C, table, n).cpu().numpy(), O.block_sparse_table(lcp_o))
    exp = O.lcp_pairs(text, p, q)
    np.testing.assert_array_equal(ans.cpu().numpy(), exp)
    np.testing.assert_array_equal(val.cpu().numpy(), exp)
    k = min(p.size, 20_000)  # the argmin oracle runs one query at a time
    ev, ea = O.rmq_argmin(lcp_o, O.inverse_suffix_array(sa_o), p[:k], q[:k])
    np.testing.assert_array_equal(val.cpu().numpy()[:k], ev)
    np.testing.assert_array_equal(arg.cpu().numpy()[:k], ea)


@pytest.mark.parametrize("total", [1, 2, 30, 31, 32, 33, 63, 64, 65, 95, 1000, 4097])
def test_block_rmq_sizes_around_the_block(L, oracle_mod, total):
    rng = np.random.default_rng(total)
    a = np.frombuffer(b"AC", np.uint8)
    l1 = int(rng.integers(0, total + 1))
    seqs = [a[rng.integers(0, 2, l1)], a[rng.integers(0, 2, total - l1)]]
    run_case(L, oracle_mod, seqs, 0, 0, all_pairs=(total + 2) <= 400)
    if total + 2 > 400:
        run_case(L, oracle_mod, seqs, 50_000, total)


def test_block_rmq_2x1M(L, oracle_mod):
    seqs, _ = gen.pair_uniform(n_each=1_000_000, plant_len=500, seed=140434494)
    run_case(L, oracle_mod, seqs, 200_000, 7)


def test_block_rmq_bad_position_is_reported(L):
    t = torch.tensor([3, 4, 3, 1], dtype=torch.uint8).cuda()
    sa = L.build_sa(t, 5)
    isa, lcp = L.lcp(t, sa)
    table = L.rmq_block_build(lcp)
    p = torch.tensor([0, 7], dtype=torch.int32).cuda()
    q = torch.tensor([2, 1], dtype=torch.int32).cuda()
    ans = L.rmq_block_query(table, lcp, isa, p, q)
    assert L.device_status() == -7  # LOR_ERR_BAD_INPUT, then cleared
    assert ans.cpu().numpy()[1] == -1
    assert L.device_status() == 0
