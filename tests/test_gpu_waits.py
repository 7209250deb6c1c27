"""The failure path of the bounded waits, exercised without a fault.

Every inter-block wait of the library (the decoupled look-back of the radix
passes and scans) gives up after a limit and records LOR_ERR_TIMEOUT instead
of spinning forever.  Here the first tile of every radix pass withholds its
look-back descriptor (a flag that nothing else sets) under a 2 ms limit, so
the tile after it must give up: the call reports LOR_ERR_TIMEOUT through
lor_device_status, every access stays in bounds, and the next call at the
default limit sorts correctly (checked against the oracle's radix sort built
from the 1-bit split of Section 4, Algorithm 1).
"""
import numpy as np
import pytest

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


def _keys(m, bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << bits, m, dtype=np.int64).astype(np.uint64)
    vals = np.arange(m, dtype=np.uint32)
    return keys, vals


def test_starved_lookback_times_out_then_recovers(L, oracle_mod):
    m, bits = 250_000, 40  # 82 tiles of 3072 keys, five 8-bit passes
    keys, vals = _keys(m, bits, 7)
    k_t = torch.from_numpy(keys.view(np.int64)).cuda()
    v_t = torch.from_numpy(vals.view(np.int32)).cuda()
    L.check_device(where="before")
    L.test_set_wait(limit_ns=2_000_000, starve_first_tile=True)
    try:
        L.radix_sort_pairs(k_t, v_t, bits)  # host-side checks pass; the device gives up
        status = L.device_status()
    finally:
        L.test_set_wait()  # the default limit, nothing starved
    assert status == L.LOR_ERR_TIMEOUT, L.status_string(status)
    assert L.device_status() == L.LOR_OK  # read and cleared

    k_t = torch.from_numpy(keys.view(np.int64)).cuda()
    v_t = torch.from_numpy(vals.view(np.int32)).cuda()
    L.radix_sort_pairs(k_t, v_t, bits)
    L.check_device(where="after the limit is restored")
    ek, ev = oracle_mod.radix_sort_split(keys, bits, values=vals.astype(np.int64))
    np.testing.assert_array_equal(k_t.cpu().numpy().view(np.uint64), ek)
    np.testing.assert_array_equal(v_t.cpu().numpy().view(np.uint32), ev.astype(np.uint32))


def test_wait_limit_arguments(L):
    with pytest.raises(L.LorError):
        L.test_set_wait(limit_ns=3_000_000_000)  # above the 2 s default
    L.test_set_wait()
