"""Continuous-batching server: requests of mixed kinds and sizes arrive
while others run; every result equals the same request computed alone
(single library call) and, for sampled requests, the oracle.  Admission
respects the device-memory budget."""
import threading
import time

import numpy as np
import pytest

import gen
from gpu_util import bits, dev, f32_matrix, host, int_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def _requests(count, seed):
    import torch
    sizes = gen.loguniform_sizes(seed, 1, count, 16, 700)
    kinds = gen.uniform_int(seed, 2, (count,), 0, 3)  # 0,1: APSP, 2: int32 product, 3: fp32 product
    reqs = []
    for i, (n, kd) in enumerate(zip(sizes, kinds)):
        n = int(n)
        if kd <= 1:
            W = gen.random_graph(seed + 10 + i, i, n, 0.1 if n > 10 else 0.5, 1, 100)
            reqs.append(("apsp", torch.from_numpy(W).pin_memory(), torch.empty((n, n), dtype=torch.int32).pin_memory()))
        else:
            sr = i % 2
            mk = int_matrix if kd == 2 else f32_matrix
            A = mk(seed + 100 + i, (n, max(1, n // 2 + 3)), sr)
            B = mk(seed + 200 + i, (A.shape[1], max(1, n - 5)), sr)
            C = torch.empty((n, B.shape[1]), dtype=torch.int32 if kd == 2 else torch.float32).pin_memory()
            reqs.append(("gemm", torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), C, sr))
    return reqs


def _alone(btas, r):
    if r[0] == "apsp":
        return host(btas.apsp(r[1].cuda()))
    return host(btas.gemm(r[1].cuda(), r[2].cuda(), r[4]))


@pytest.mark.parametrize("whole", [True, False])
def test_mixed_arrivals_match_single_calls(btas, oracle_mod, whole):
    """whole=True: APSP requests with n <= 1024 are solved in one unit (the
    one-block or the cooperative kernel); whole=False
    (BTAS_SERVER_NO_WHOLE=1): one squaring per step, through the persistent
    tile-task kernel."""
    import os
    reqs = _requests(40, 7)
    if not whole:
        os.environ["BTAS_SERVER_NO_WHOLE"] = "1"
    try:
        srv = btas.Server(40 << 30)
    finally:
        os.environ.pop("BTAS_SERVER_NO_WHOLE", None)
    tickets = []

    def producer():
        for i, r in enumerate(reqs):
            if r[0] == "apsp":
                tickets.append(srv.submit_apsp(r[1], r[2]))
            else:
                tickets.append(srv.submit_gemm(r[1], r[2], r[3], r[4]))
            time.sleep(0.0005 * (i % 3))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    srv.wait_all(120)
    for t in tickets:
        st = srv.poll(t)
        assert st["state"] == 2 and st["t_done"] >= st["t_admit"] >= st["t_submit"]
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["bytes_in_use"] == 0
    srv.close()
    for i, r in enumerate(reqs):
        out = (r[2] if r[0] == "apsp" else r[3]).numpy()
        np.testing.assert_array_equal(bits(out), bits(_alone(btas, r)), err_msg=f"request {i} {r[0]}")
        if i % 7 == 0:
            if r[0] == "apsp":
                np.testing.assert_array_equal(out, oracle_mod.floyd_warshall(r[1].numpy()))
            else:
                np.testing.assert_array_equal(bits(out), bits(oracle_mod.tgemm(r[4], r[1].numpy(), r[2].numpy())))


def test_small_budget_queues_and_rejects(btas):
    import paper_1701_04733_gb300 as b_mod
    import torch
    reqs = _requests(12, 11)
    # about two of the larger requests fit at a time
    srv = btas.Server(16 << 20)
    tickets = []
    for r in reqs:
        if r[0] == "apsp":
            tickets.append(srv.submit_apsp(r[1], r[2]))
        else:
            tickets.append(srv.submit_gemm(r[1], r[2], r[3], r[4]))
    srv.wait_all(120)
    for r in reqs:
        out = (r[2] if r[0] == "apsp" else r[3]).numpy()
        np.testing.assert_array_equal(bits(out), bits(_alone(btas, r)))
    big = torch.zeros((2048, 2048), dtype=torch.int32)
    with pytest.raises(b_mod.BtasError) as ei:
        srv.submit_apsp(big, big.clone())
    assert ei.value.status == 6
    srv.close()


def test_whole_solve_domain_violation_fails_alone(btas, oracle_mod):
    """An APSP request whose W is outside the domain (a negative weight) ends
    in the failed state; the requests around it are unaffected.  With whole
    solves off (BTAS_SERVER_NO_WHOLE=1) every request runs squaring by
    squaring, so the bad request is caught by the domain scan of its first
    squaring step (test_whole_solve_domain_check_alone covers the
    whole-solve check)."""
    import os
    import torch
    good = gen.random_graph(31, 1, 300, 0.05, 1, 100)
    bad = good.copy()
    bad[4, 9] = -2
    large = gen.random_graph(32, 1, 1900, 0.01, 1, 100)
    bufs = [(torch.from_numpy(w).pin_memory(), torch.zeros(w.shape, dtype=torch.int32).pin_memory())
            for w in (good, bad, large, good[:100, :100].copy())]
    bufs[1][1].fill_(77)
    os.environ["BTAS_SERVER_NO_WHOLE"] = "1"
    try:
        srv = btas.Server(8 << 30)
    finally:
        os.environ.pop("BTAS_SERVER_NO_WHOLE", None)
    tickets = [srv.submit_apsp(W, D) for W, D in bufs]
    srv.wait_all(120)
    states = [srv.poll(t)["state"] for t in tickets]
    srv.close()
    assert states == [2, 3, 2, 2]
    assert (bufs[1][1].numpy() == 77).all()  # a failed request leaves D alone
    np.testing.assert_array_equal(bufs[0][1].numpy(), oracle_mod.floyd_warshall(good))
    np.testing.assert_array_equal(bufs[2][1].numpy(), host(btas.apsp(dev(large))))
    np.testing.assert_array_equal(bufs[3][1].numpy(), oracle_mod.floyd_warshall(good[:100, :100].copy()))


def test_whole_solve_domain_check_alone(btas, oracle_mod):
    """With no other pending work the bad request is solved whole, and the
    whole-solve kernel's own domain check fails it."""
    import torch
    good = gen.random_graph(33, 1, 300, 0.05, 1, 100)
    bad = good.copy()
    bad[7, 2] = -5
    bufs = [(torch.from_numpy(w).pin_memory(), torch.zeros(w.shape, dtype=torch.int32).pin_memory())
            for w in (bad, good)]
    bufs[0][1].fill_(77)
    srv = btas.Server(8 << 30)
    tickets = [srv.submit_apsp(W, D) for W, D in bufs]
    srv.wait_all(120)
    states = [srv.poll(t)["state"] for t in tickets]
    srv.close()
    assert states == [3, 2]
    assert (bufs[0][1].numpy() == 77).all()  # a failed request leaves D alone
    np.testing.assert_array_equal(bufs[1][1].numpy(), oracle_mod.floyd_warshall(good))


def test_chunked_steps_match_single_calls(btas, oracle_mod):
    """A step cap far below one unit (BTAS_SERVER_STEP_TERMS=5e7) makes every
    larger product and squaring run as chunks of its output tiles over
    several steps, while small units join each step.  Whole solves are off,
    so every APSP squaring goes through the persistent kernel: the first
    squaring picks packed or int32 on the device from W's largest weight
    (weights up to 100, and up to 20000 where 2 * max >= 0x7FFF).  A request
    outside the domain fails after the chunk that scanned it.  Every other
    result equals its single call."""
    import os
    import torch
    reqs = _requests(24, 19)
    heavy = gen.random_graph(41, 1, 600, 0.02, 1, 20000)
    reqs.append(("apsp", torch.from_numpy(heavy).pin_memory(), torch.empty((600, 600), dtype=torch.int32).pin_memory()))
    bad = gen.random_graph(42, 1, 500, 0.05, 1, 100)
    bad[3, 3] = 5  # non-zero diagonal
    bad_t = torch.from_numpy(bad).pin_memory()
    bad_out = torch.full((500, 500), 77, dtype=torch.int32).pin_memory()
    os.environ["BTAS_SERVER_STEP_TERMS"] = "5e7"
    os.environ["BTAS_SERVER_NO_WHOLE"] = "1"
    try:
        srv = btas.Server(40 << 30)
    finally:
        os.environ.pop("BTAS_SERVER_STEP_TERMS", None)
        os.environ.pop("BTAS_SERVER_NO_WHOLE", None)
    tickets = []
    for i, r in enumerate(reqs):
        if r[0] == "apsp":
            tickets.append(srv.submit_apsp(r[1], r[2]))
        else:
            tickets.append(srv.submit_gemm(r[1], r[2], r[3], r[4]))
        if i == 5:
            bad_ticket = srv.submit_apsp(bad_t, bad_out)
    srv.wait_all(300)
    assert [srv.poll(t)["state"] for t in tickets] == [2] * len(tickets)
    assert srv.poll(bad_ticket)["state"] == 3
    stats = srv.stats()
    srv.close()
    # the 600-vertex graph alone needs 25 output tiles of 128^2 x 600 terms per
    # squaring: at most 5 per step under the cap, so its squarings span steps
    assert stats["steps"] >= 10
    assert (bad_out.numpy() == 77).all()
    for i, r in enumerate(reqs):
        out = (r[2] if r[0] == "apsp" else r[3]).numpy()
        np.testing.assert_array_equal(bits(out), bits(_alone(btas, r)), err_msg=f"request {i} {r[0]}")
    np.testing.assert_array_equal(reqs[-1][2].numpy(), oracle_mod.floyd_warshall(heavy))


def test_bulk_lane_matches_single_calls(btas, oracle_mod):
    """Large requests take the bulk lane (forced here down to 2e7 terms with
    BTAS_SERVER_BULK_TERMS) and run through the single calls on their own
    thread and stream, concurrently with the step loop's batched work.  Every
    result equals its single call; an APSP request above the cooperative
    kernel's size limit (always bulk) outside the weight domain fails and
    leaves D alone."""
    import os
    import torch
    reqs = _requests(30, 23)
    bad = gen.random_graph(43, 1, 1900, 0.01, 1, 100)
    bad[10, 11] = -1
    bad_t = torch.from_numpy(bad).pin_memory()
    bad_out = torch.full((1900, 1900), 77, dtype=torch.int32).pin_memory()
    os.environ["BTAS_SERVER_BULK_TERMS"] = "2e7"
    try:
        srv = btas.Server(40 << 30)
    finally:
        os.environ.pop("BTAS_SERVER_BULK_TERMS", None)
    tickets = []
    for i, r in enumerate(reqs):
        if r[0] == "apsp":
            tickets.append(srv.submit_apsp(r[1], r[2]))
        else:
            tickets.append(srv.submit_gemm(r[1], r[2], r[3], r[4]))
        if i == 3:
            bad_ticket = srv.submit_apsp(bad_t, bad_out)
    srv.wait_all(300)
    assert [srv.poll(t)["state"] for t in tickets] == [2] * len(tickets)
    assert srv.poll(bad_ticket)["state"] == 3
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()
    assert (bad_out.numpy() == 77).all()
    for i, r in enumerate(reqs):
        out = (r[2] if r[0] == "apsp" else r[3]).numpy()
        np.testing.assert_array_equal(bits(out), bits(_alone(btas, r)), err_msg=f"request {i} {r[0]}")
        if i % 5 == 0 and r[0] == "gemm":
            np.testing.assert_array_equal(bits(out), bits(oracle_mod.tgemm(r[4], r[1].numpy(), r[2].numpy())))
