"""One reference against many queries (lor_multi_query_overlap) against the
oracle: every query's length, query offset and reference offset, exactly."""
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


def run(L, ref, qs):
    ref_dev = torch.from_numpy(np.array(ref, dtype=np.uint8)).cuda()
    flat = np.concatenate(qs) if sum(len(q) for q in qs) else np.zeros(0, np.uint8)
    q_dev = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.uint8)).cuda()
    out = L.multi_query_overlap(ref_dev, q_dev, [len(q) for q in qs])
    L.check_device(where="multi query")
    return out.cpu().numpy()[:, :3].astype(np.int64)


def test_multi_query_small_cases(L, oracle_mod):
    rng = np.random.default_rng(21)
    A = np.frombuffer(b"ACGT", np.uint8)
    refs = [A[rng.integers(0, 4, 2000)], np.frombuffer(b"ACACACACAC" * 40, np.uint8),
            np.frombuffer(b"G", np.uint8), np.zeros(0, np.uint8)]
    for ref in refs:
        qs = [A[rng.integers(0, 4, int(rng.integers(0, 80)))] for _ in range(300)]
        qs += [np.frombuffer(b"CA" * 9, np.uint8), np.zeros(0, np.uint8), np.frombuffer(b"T", np.uint8),
               np.frombuffer(b"acgt", np.uint8).copy()]
        if ref.size > 300:
            qs += [ref[100:300].copy(), ref[:50].copy(), ref[-70:].copy()]
        got = run(L, ref, qs)
        upper = [np.frombuffer(bytes(q).upper(), np.uint8) for q in qs]
        np.testing.assert_array_equal(got, oracle_mod.multi_query(ref, upper))


def test_multi_query_noncoding_reference_thousands_of_queries(L, oracle_mod):
    ref, qs = gen.multi_query(ref_len=200_000, nq=3000, lo=50, hi=3000, seed=140434495)
    got = run(L, ref, qs)
    np.testing.assert_array_equal(got, oracle_mod.multi_query(ref, qs))
    assert (got[:, 0] >= 20).mean() > 0.9  # reads and planted pieces are found


def test_multi_query_many_tiles_and_long_matches(L, oracle_mod):
    ref, qs = gen.multi_query(ref_len=2_000_000, nq=400, lo=1000, hi=60_000, seed=140434496)
    qs += [ref[5000:45000].copy()]  # an exact 40,000-base read
    got = run(L, ref, qs)
    np.testing.assert_array_equal(got, oracle_mod.multi_query(ref, qs))
    assert got[-1, 0] == 40_000
