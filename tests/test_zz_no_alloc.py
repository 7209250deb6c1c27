"""The suffix-array entry point for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc to size a workspace -- for example a
plugin running inside an application that owns the device memory pool, or a
callback that must not block on the allocator.  lor_build_sa_noalloc serves
them with scratch held inside the library.  These checks call it through the
C ABI and compare its suffix arrays with those of lor_build_sa (caller
workspace) and with the CPU oracle's (suffixes sorted by direct comparison):
equal element by element, the exactness every integer output of this library
is held to.  Two different texts go through it back to back, because every
call shares the same scratch and inherits what the previous call left there;
the first one is the largest accepted size.  One symbol more must be refused
before any device work, and bad arguments are reported as lor_build_sa
reports them.

The file name makes pytest collect it last.
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
    from paper_1404_3448_gb300 import lor
    lor.load()
    return lor


def _encoded(L, seqs):
    lens = [len(s) for s in seqs]
    ascii_dev = torch.from_numpy(np.concatenate(seqs)).cuda()
    text, _, sigma = L.encode_concat(ascii_dev, lens)
    return text, sigma


def test_noalloc_matches_workspace_path_on_two_calls_in_a_row(L, oracle_mod):
    max_n = 262144
    half = (max_n - 2) // 2
    seqs_a, _ = gen.pair_uniform(n_each=half, plant_len=300, seed=9001)
    seqs_b, _ = gen.pair_noncoding(n_each=50_000, seed=9002, shared_len=3000, core=800)
    text_a, sig_a = _encoded(L, seqs_a)
    text_b, sig_b = _encoded(L, seqs_b)
    assert text_a.numel() == max_n

    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for text, sigma in ((text_a, sig_a), (text_b, sig_b)):
        sa = torch.full((text.numel(),), -1, dtype=torch.int32, device="cuda")
        rc = L.lor_build_sa_noalloc(text.data_ptr(), text.numel(), sigma, sa.data_ptr(), stream)
        assert rc == L.LOR_OK, L.status_string(rc)
        assert L.device_status() == L.LOR_OK
        got.append(sa)

    for sa, (text, sigma), seqs in zip(got, ((text_a, sig_a), (text_b, sig_b)), (seqs_a, seqs_b)):
        ref = L.build_sa(text, sigma)
        L.check_device()
        assert torch.equal(sa, ref)
        o_text, _, _ = oracle_mod.encode_concat(seqs)
        np.testing.assert_array_equal(text.cpu().numpy(), o_text)
        np.testing.assert_array_equal(sa.cpu().numpy(), oracle_mod.suffix_array(o_text))


def test_noalloc_refuses_texts_above_its_limit(L):
    text = torch.ones(16, dtype=torch.uint8, device="cuda")
    sa = torch.empty(16, dtype=torch.int32, device="cuda")
    rc = L.lor_build_sa_noalloc(text.data_ptr(), 262145, 7, sa.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == L.LOR_ERR_TOO_LARGE


def test_noalloc_checks_arguments_before_its_size_limit(L):
    stream = torch.cuda.current_stream().cuda_stream
    sa = torch.empty(16, dtype=torch.int32, device="cuda")
    # a null text is an invalid argument whatever n is, as for lor_build_sa
    assert L.lor_build_sa_noalloc(None, 262145, 7, sa.data_ptr(), stream) == L.LOR_ERR_INVALID_ARG
    assert L.lor_build_sa_noalloc(None, 100, 7, sa.data_ptr(), stream) == L.LOR_ERR_INVALID_ARG
    text = torch.ones(16, dtype=torch.uint8, device="cuda")
    assert L.lor_build_sa_noalloc(text.data_ptr(), 16, 1, sa.data_ptr(), stream) == L.LOR_ERR_INVALID_ARG
