"""btas_apsp_noalloc: APSP for callers that cannot allocate device memory
when they call (for example, a process whose own pool already holds the
device's free memory, or a latency-critical loop that must not allocate).

The entry point keeps its scratch in a fixed device array instead of
allocating.  These checks call it through the C ABI and compare it with
btas_apsp, the allocating entry point, on two calls in a row: the second call
starts from the scratch the first one left behind.  Distances are integers,
so the comparison is exact.  Collected last, so a failure here comes after
every other test has run."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def _both(btas, W):
    import torch
    n = W.shape[0]
    Wd = torch.from_numpy(W).cuda()
    ref = torch.empty_like(Wd)
    out = torch.full_like(Wd, -7)
    stream = torch.cuda.current_stream().cuda_stream
    assert btas.btas_apsp(n, Wd.data_ptr(), ref.data_ptr(), stream) == 0, btas.last_error()
    assert btas.btas_apsp_noalloc(n, Wd.data_ptr(), out.data_ptr(), stream) == 0, btas.last_error()
    torch.cuda.synchronize()
    return ref.cpu().numpy(), out.cpu().numpy()


def test_two_calls_match_allocating_entry_point(btas):
    W1 = gen.random_graph(gen.BASE_SEED, 71, 1000, 0.05, 1, 100)
    W2 = gen.random_graph(gen.BASE_SEED, 72, 777, 0.1, 1, 1000)
    ref1, out1 = _both(btas, W1)
    np.testing.assert_array_equal(out1, ref1)
    ref2, out2 = _both(btas, W2)
    np.testing.assert_array_equal(out2, ref2)


def test_tiled_fallback(btas):
    """The tiled int32 squarings, which serve where a cooperative launch is
    refused (forced here with BTAS_APSP_NO_MID=1), out of place and in place,
    twice in a row."""
    import os
    import torch
    os.environ["BTAS_APSP_NO_MID"] = "1"
    try:
        for n, seed in ((1000, 79), (333, 80)):
            W = gen.random_graph(gen.BASE_SEED, seed, n, 0.05, 1, 100)
            ref, out = _both(btas, W)
            np.testing.assert_array_equal(out, ref)
            t = torch.from_numpy(W).cuda()
            stream = torch.cuda.current_stream().cuda_stream
            assert btas.btas_apsp_noalloc(n, t.data_ptr(), t.data_ptr(), stream) == 0
            torch.cuda.synchronize()
            np.testing.assert_array_equal(t.cpu().numpy(), ref)
    finally:
        del os.environ["BTAS_APSP_NO_MID"]


def test_in_place_and_size_limit(btas):
    import torch
    W = gen.random_graph(gen.BASE_SEED, 73, 300, 0.05, 1, 50)
    ref, _ = _both(btas, W)
    t = torch.from_numpy(W).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    assert btas.btas_apsp_noalloc(300, t.data_ptr(), t.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(t.cpu().numpy(), ref)
    # beyond the fixed scratch: rejected on the host, nothing enqueued
    assert btas.btas_apsp_noalloc(1025, t.data_ptr(), t.data_ptr(), stream) == 1
    assert "1024" in btas.last_error()


def test_small_and_mid_sizes(btas):
    """The one-block (smallest n) and cooperative (up to n = 1024) kernels
    behind the allocation-free entry point, out of place and in place."""
    import torch
    for n, seed in ((3, 74), (100, 75), (129, 76), (512, 77)):
        W = gen.random_graph(gen.BASE_SEED, seed, n, 0.5 if n < 8 else 0.05, 1, 100)
        ref, out = _both(btas, W)
        np.testing.assert_array_equal(out, ref)
        t = torch.from_numpy(W).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        assert btas.btas_apsp_noalloc(n, t.data_ptr(), t.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), ref)
