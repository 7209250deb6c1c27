"""The request server (lor_server_*) against the oracle and against itself.

Every request's record, positions and LCP-query answers must equal what the
oracle computes for that pair alone (its own text S1#S2$), and must be the
same whether the request ran alone or batched with others that arrived around
it.  Admission under a tight device budget, rejection of oversized pairs and
the release of resident state are checked too.
"""
import time

import numpy as np
import pytest

import lor_inputs as gen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NQ = 16


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1404_3448_gb300 as lor
    lor.load()
    return lor


def pair_text(O, a, b):
    text, starts, _ = O.encode_concat([a, b])
    return text, starts


def expect(O, a, b, p, q):
    text, starts = pair_text(O, a, b)
    sa = O.suffix_array(text)
    lcp = O.lcp_array(text, sa)
    ov = O.longest_overlap(text, sa, lcp, starts)
    return ov, O.lcp_pairs(text, p, q)


def queries_for(a, b, seed):
    """16 (p, q) suffix pairs of S1#S2$: uniform, plus p == q, the
    terminators and the last suffix."""
    n = len(a) + len(b) + 2
    rng = np.random.default_rng(seed)
    p = rng.integers(0, n, size=NQ).astype(np.int32)
    q = rng.integers(0, n, size=NQ).astype(np.int32)
    p[0] = q[0] = n // 2
    p[1], q[1] = len(a), n - 1
    p[2], q[2] = 0, n - 1
    return p, q


def assert_record(got, exp, tag):
    for k in ("length", "rank", "seq_a", "pos_a", "seq_b", "pos_b"):
        assert got[k] == exp[k], (tag, k, got[k], exp[k])
    assert got["n_pos"] == len(exp["positions"]), tag
    np.testing.assert_array_equal(got["positions"], exp["positions"], err_msg=str(tag))


def drain(srv, want, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < want:
        for r in srv.poll(timeout_ms=50):
            got[r["id"]] = r
        assert time.time() - t0 < timeout_s, f"only {len(got)} of {want} results"
    return got


def serve_mix(L, pairs, workers=2, max_pairs=7, budget=8 << 30, gap_s=0.0005, seed=0):
    """Submit all pairs with small random gaps, then query every request and
    release it.  Returns per-request (record, answers) in submit order."""
    rng = np.random.default_rng(seed)
    res, ids = [], []
    with L.Server(budget, workers=workers, max_batch_pairs=max_pairs) as srv:
        for i, (a, b) in enumerate(pairs):
            ids.append(srv.submit(a, b, tag=i))
            if gap_s:
                time.sleep(float(rng.uniform(0, gap_s)))
        got = drain(srv, len(pairs))
        for i, rid in enumerate(ids):
            r = got[rid]
            assert r["status"] == 0 and r["tag"] == i
            p, q = queries_for(*pairs[i], seed=1000 + i)
            res.append((r, srv.query(rid, p, q)))
        for rid in ids:
            srv.release(rid)
        st = srv.stats()
        assert st["in_use_bytes"] == 0 and st["completed"] == len(pairs) and st["released"] == len(pairs)
        assert st["queries"] == NQ * len(pairs)
    return res


def mixed_pairs():
    pairs = [list(pr) for pr in gen.pair_batch(npairs=36, lo=300, hi=40_000, seed=140434491)]
    cases = [v for v in gen.degenerate_cases().values() if len(v) == 2]
    pairs += [list(c) for c in cases]
    pairs.append([np.zeros(0, np.uint8), np.frombuffer(b"ACGT", np.uint8).copy()])
    return pairs


def test_serve_mix_equals_alone_and_oracle(L, oracle_mod):
    pairs = mixed_pairs()
    mix = serve_mix(L, pairs, workers=2, max_pairs=7)
    alone = serve_mix(L, pairs, workers=1, max_pairs=1, gap_s=0)
    assert max(r["batch_pairs"] for r, _ in mix) > 1, "the mix never batched two requests"
    assert all(r["batch_pairs"] == 1 for r, _ in alone)
    for i, (a, b) in enumerate(pairs):
        (rm, qm), (ra, qa) = mix[i], alone[i]
        p, q = queries_for(a, b, seed=1000 + i)
        ov, lq = expect(oracle_mod, a, b, p, q)
        assert_record(rm, ov, ("mix", i))
        assert_record(ra, ov, ("alone", i))
        np.testing.assert_array_equal(qm, lq, err_msg=f"mix queries {i}")
        np.testing.assert_array_equal(qa, lq, err_msg=f"alone queries {i}")


def test_serve_admission_under_tight_budget(L, oracle_mod):
    """A reservation of about two single-pair batches: requests wait for
    memory (results and resident state are released as they arrive) and all
    finish with the oracle's results."""
    pairs = [list(pr) for pr in gen.pair_batch(npairs=14, lo=20_000, hi=200_000, seed=140434492)]
    need = max(sum(L.server_batch_bytes([len(a), len(b)])) for a, b in pairs)
    budget = int(need * 2.5) + (8 << 20)
    with L.Server(budget, workers=3, max_batch_pairs=4) as srv:
        ids = {srv.submit(a, b, tag=i): i for i, (a, b) in enumerate(pairs)}
        seen = 0
        t0 = time.time()
        while seen < len(pairs):
            for r in srv.poll(timeout_ms=50):
                i = ids[r["id"]]
                assert r["status"] == 0
                p, q = queries_for(*pairs[i], seed=i)
                ov, lq = expect(oracle_mod, *pairs[i], p, q)
                assert_record(r, ov, i)
                np.testing.assert_array_equal(srv.query(r["id"], p, q), lq)
                srv.release(r["id"])
                seen += 1
            assert time.time() - t0 < 120, f"only {seen} of {len(pairs)} results"
        st = srv.stats()
        assert st["peak_bytes"] <= st["reserved_bytes"] <= budget
        assert st["in_use_bytes"] == 0 and st["pending"] == 0 and st["in_flight"] == 0


def test_serve_rejections(L):
    a = np.frombuffer(b"ACGTACGTAC", np.uint8).copy()
    with L.Server(64 << 20, workers=1, max_batch_pairs=4) as srv:
        big = np.zeros(8 << 20, np.uint8) + ord("A")
        with pytest.raises(L.LorError) as e:
            srv.submit(big, big)
        assert e.value.status == L.lor.LOR_ERR_TOO_LARGE
        rid = srv.submit(a, a)
        with pytest.raises(L.LorError):
            srv.release(rid + 1000)  # unknown id
        r = drain(srv, 1)[rid]
        assert r["status"] == 0 and r["length"] == 10
        n = 2 * len(a) + 2
        with pytest.raises(L.LorError):
            srv.query(rid, np.array([n], np.int32), np.array([0], np.int32))
        assert srv.query(rid, np.array([0, 3], np.int32), np.array([11, 3], np.int32)).tolist() == [10, n - 3]
        srv.release(rid)
        with pytest.raises(L.LorError):
            srv.query(rid, np.array([0], np.int32), np.array([1], np.int32))  # released


def test_serve_many_small_requests_match_batched_path(L):
    pairs = [list(gen.fuzz_sequences(9000 + i, nseq=2, max_len=[8, 300, 3000][i % 3])) for i in range(300)]
    mix = serve_mix(L, pairs, workers=3, max_pairs=512, gap_s=0)
    lens = [len(s) for pr in pairs for s in pr]
    b = L.lor.Batch(lens, pos_cap=1 << 22)
    b.run(torch.from_numpy(np.concatenate([s for pr in pairs for s in pr])).cuda())
    L.check_device(where="batch")
    ref = b.results()
    for i, (r, _) in enumerate(mix):
        assert_record(r, ref[i], i)


def test_serve_pairs_up_to_4M_bases(L, oracle_mod):
    """Served requests at the sizes of the served workload (per-sequence
    lengths log-uniform in [1k, 4M], two pairs near 4M bases each): each
    request's record, positions and 16 follow-up answers equal the oracle's,
    alone and in a mix where batches of several pairs run at once."""
    pairs = [list(pr) for pr in gen.pair_batch(npairs=8, lo=1_000, hi=4_000_000, seed=140434493)]
    pairs += [list(pr) for pr in gen.pair_batch(npairs=2, lo=3_500_000, hi=4_000_000, seed=140434494)]
    assert max(len(a) + len(b) for a, b in pairs) > 7_000_000
    queries = [queries_for(a, b, seed=1000 + i) for i, (a, b) in enumerate(pairs)]
    exp = oracle_mod.pair_overlaps(pairs, queries=queries)
    mix = serve_mix(L, pairs, workers=2, max_pairs=4, budget=24 << 30, gap_s=0)
    alone = serve_mix(L, pairs, workers=1, max_pairs=1, budget=24 << 30, gap_s=0)
    assert max(r["batch_pairs"] for r, _ in mix) > 1, "the mix never batched two requests"
    for i in range(len(pairs)):
        (rm, qm), (ra, qa) = mix[i], alone[i]
        assert_record(rm, exp[i], ("mix", i))
        assert_record(ra, exp[i], ("alone", i))
        np.testing.assert_array_equal(qm, exp[i]["answers"], err_msg=f"mix queries {i}")
        np.testing.assert_array_equal(qa, exp[i]["answers"], err_msg=f"alone queries {i}")


def test_serve_bad_request_fails_alone(L, oracle_mod):
    """One request holds a byte that is not a base.  Two workers run batches
    at once, each recording device errors in a status slot of its own: the
    bad request fails with LOR_ERR_BAD_SYMBOL, and every other request --
    including those batched with it, which are run again alone -- succeeds
    with the oracle's results.  Nothing leaks into lor_device_status."""
    pairs = [list(pr) for pr in gen.pair_batch(npairs=40, lo=300, hi=30_000, seed=140434495)]
    bad = 17
    pairs[bad][0] = pairs[bad][0].copy()
    pairs[bad][0][len(pairs[bad][0]) // 2] = ord("N")
    exp = oracle_mod.pair_overlaps([pr for i, pr in enumerate(pairs) if i != bad])
    exp.insert(bad, None)
    L.check_device(where="before the server")
    with L.Server(4 << 30, workers=2, max_batch_pairs=8) as srv:
        ids = [srv.submit(a, b, tag=i) for i, (a, b) in enumerate(pairs)]
        got = drain(srv, len(pairs))
        for i, rid in enumerate(ids):
            r = got[rid]
            if i == bad:
                assert r["status"] == L.lor.LOR_ERR_BAD_SYMBOL, r["status"]
                continue
            assert r["status"] == 0, (i, r["status"])
            assert_record(r, exp[i], i)
            srv.release(rid)
        assert max(got[rid]["batch_pairs"] for rid in ids) > 1, "no request was batched"
    assert L.device_status() == 0

