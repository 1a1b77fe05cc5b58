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
        for n, seed in ((1000, 79), (333, 80), (1024, 81)):
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
    behind the allocation-free entry point, out of place and in place.
    n = 1024 fills the fixed array exactly (three iterates plus the barrier
    and status words)."""
    import torch
    for n, seed in ((3, 74), (100, 75), (129, 76), (512, 77), (1024, 78)):
        W = gen.random_graph(gen.BASE_SEED, seed, n, 0.5 if n < 8 else 0.05, 1, 100)
        ref, out = _both(btas, W)
        np.testing.assert_array_equal(out, ref)
        t = torch.from_numpy(W).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        assert btas.btas_apsp_noalloc(n, t.data_ptr(), t.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        np.testing.assert_array_equal(t.cpu().numpy(), ref)


def _status(btas):
    import ctypes
    import torch
    sq = ctypes.c_int(-1)
    st = btas.btas_apsp_noalloc_status(torch.cuda.current_stream().cuda_stream, ctypes.addressof(sq))
    return st, sq.value


def test_status_reports_squarings(btas):
    """The status query reads what the last call left in the fixed array: for
    every regime (one block, cooperative, tiled fallback) the squarings that
    changed D equal those btas_apsp reports for the same graph."""
    import os
    import torch
    for n, seed, no_mid in ((40, 82, False), (700, 83, False), (700, 83, True)):
        W = gen.random_graph(gen.BASE_SEED, seed, n, 0.05, 1, 100)
        Wd = torch.from_numpy(W).cuda()
        ref, info = btas.apsp(Wd, info=True)
        out = torch.empty_like(Wd)
        if no_mid:
            os.environ["BTAS_APSP_NO_MID"] = "1"
        try:
            assert btas.btas_apsp_noalloc(n, Wd.data_ptr(), out.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream) == 0
        finally:
            os.environ.pop("BTAS_APSP_NO_MID", None)
        st, sq = _status(btas)
        assert st == 0, btas.last_error()
        assert sq == info["squarings"]
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_status_reports_domain_violation(btas):
    """A weight outside the domain: the kernel leaves D unwritten and the
    status query returns BTAS_ERR_ARG; the next call succeeds."""
    import torch
    for n, seed in ((40, 84), (300, 85)):
        W = gen.random_graph(gen.BASE_SEED, seed, n, 0.05, 1, 100)
        bad = W.copy()
        bad[1, 2] = -5
        out = torch.full((n, n), 41, dtype=torch.int32, device="cuda")
        b = torch.from_numpy(bad).cuda()
        stream = torch.cuda.current_stream().cuda_stream
        assert btas.btas_apsp_noalloc(n, b.data_ptr(), out.data_ptr(), stream) == 0
        st, _ = _status(btas)
        assert st == 1 and "domain" in btas.last_error()
        assert (out.cpu().numpy() == 41).all()
        ref, got = _both(btas, W)
        np.testing.assert_array_equal(got, ref)
        assert _status(btas)[0] == 0


def test_status_reports_barrier_timeout(btas):
    """Failure detection without a fault: with BTAS_MID_WITHHOLD=1 one block
    of the cooperative kernel never reaches its first grid barrier, the other
    blocks' bounded waits expire (about 2 s), D is left unwritten, and the
    status query returns BTAS_ERR_TIMEOUT.  The next call on the same context
    succeeds."""
    import os
    import torch
    n = 300
    W = gen.random_graph(gen.BASE_SEED, 86, n, 0.05, 1, 100)
    Wd = torch.from_numpy(W).cuda()
    out = torch.full((n, n), 41, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    os.environ["BTAS_MID_WITHHOLD"] = "1"
    try:
        assert btas.btas_apsp_noalloc(n, Wd.data_ptr(), out.data_ptr(), stream) == 0
    finally:
        del os.environ["BTAS_MID_WITHHOLD"]
    st, _ = _status(btas)
    assert st == 5, btas.last_error()
    assert (out.cpu().numpy() == 41).all()
    ref, got = _both(btas, W)
    np.testing.assert_array_equal(got, ref)
    assert _status(btas)[0] == 0
