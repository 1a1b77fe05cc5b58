"""Batched persistent launch (many APSP solves and tropical products of
uneven sizes in one kernel): every instance's result is bit-identical to the
single call and to the oracle; graph replay and the plain launch agree; a
withheld dependency ends in BTAS_ERR_TIMEOUT (bounded device wait) and leaves
the context usable."""
import os

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


def _mixed(btas, seed=0):
    import torch
    sizes = [1, 2, 3, 5, 31, 64, 100, 129, 200, 257, 300, 411]
    apsp = []
    for i, n in enumerate(sizes):
        W = gen.random_graph(seed + 500 + i, i, n, 0.1 if n > 8 else 0.5, 1, 100)
        apsp.append((W, dev(W), torch.empty((n, n), dtype=torch.int32, device="cuda")))
    gemm = []
    shapes = [(1, 1, 1), (7, 5, 3), (130, 129, 77), (256, 300, 200), (33, 400, 129)]
    for i, (m, n, k) in enumerate(shapes):
        for dt, sr, tb in (("f32", 1, False), ("i32", 0, True), ("f32", 0, True), ("i32", 1, False)):
            mk = int_matrix if dt == "i32" else f32_matrix
            A = mk(seed + 900 + i, (m, k), sr)
            B = mk(seed + 950 + i, (k, n), sr)
            Bd = dev(np.ascontiguousarray(B.T)) if tb else dev(B)
            C = torch.empty((m, n), dtype=torch.int32 if dt == "i32" else torch.float32, device="cuda")
            gemm.append((A, B, dev(A), Bd, C, sr, tb))
    return apsp, gemm


class _tile:
    """BTAS_BATCH_TILE for the plans built inside (None: the default)."""

    def __init__(self, tile):
        self.tile = tile

    def __enter__(self):
        if self.tile:
            os.environ["BTAS_BATCH_TILE"] = self.tile

    def __exit__(self, *a):
        os.environ.pop("BTAS_BATCH_TILE", None)


@pytest.mark.parametrize("tile", [None, "64"])
@pytest.mark.parametrize("graph", [True, False])
def test_mixed_batch_matches_single_calls_and_oracle(btas, oracle_mod, graph, tile):
    """Every instance against the oracle and the single call, with the
    default 128 x 128 output tile and with the 64 x 64 tile (4 x 4 outputs
    per thread) for every instance."""
    with _tile(tile):
        _mixed_batch_check(btas, oracle_mod, graph)


def _mixed_batch_check(btas, oracle_mod, graph):
    import torch
    apsp, gemm = _mixed(btas)
    b = btas.Batch(graph=graph)
    for W, Wd, D in apsp:
        b.add_apsp(Wd, D)
    for A, B, Ad, Bd, C, sr, tb in gemm:
        b.add_gemm(Ad, Bd, C, sr, trans_b=tb)
    for rep in range(2):  # second launch replays the plan (graph)
        for _, _, D in apsp:
            D.fill_(-5)
        for g in gemm:
            g[4].fill_(-5)
        b.launch()
        b.wait()
        for W, Wd, D in apsp:
            ref = oracle_mod.floyd_warshall(W)
            np.testing.assert_array_equal(host(D), ref, err_msg=f"apsp n={W.shape[0]} rep={rep}")
            np.testing.assert_array_equal(host(D), host(btas.apsp(Wd)))
        for A, B, Ad, Bd, C, sr, tb in gemm:
            ref = oracle_mod.tgemm(sr, A, B)
            np.testing.assert_array_equal(bits(host(C)), bits(ref), err_msg=f"gemm {A.shape}x{B.shape} sr={sr}")
    assert b.tasks > 0
    b.close()


def test_batch_of_config_sizes(btas, oracle_mod):
    """64 graphs with n uniform in [32, 1024], p = 0.1, w in [1, 100] (a slice
    of the 512-graph batched workload); 8 sampled instances vs Dijkstra rows,
    all of them vs the single-call path."""
    import torch
    sizes = gen.graph_sizes(gen.BASE_SEED, 40, 64, 32, 1024)
    b = btas.Batch()
    items = []
    for i, n in enumerate(sizes):
        W = gen.random_graph(gen.BASE_SEED, 1000 + i, int(n), 0.1, 1, 100)
        Wd = dev(W)
        D = torch.empty_like(Wd)
        b.add_apsp(Wd, D)
        items.append((W, Wd, D))
    b.launch()
    b.wait()
    for i, (W, Wd, D) in enumerate(items):
        np.testing.assert_array_equal(host(D), host(btas.apsp(Wd, flags=0x2 | 1)))
        if i % 8 == 0:
            srcs = gen.sample_indices(gen.BASE_SEED, 41 + i, 16, W.shape[0])
            np.testing.assert_array_equal(host(D)[srcs], oracle_mod.dijkstra_rows(W, srcs))
    b.close()


@pytest.mark.parametrize("tile", [None, "64"])
def test_certificate_tasks(btas, oracle_mod, tile):
    """The batched APSP's closure certificate: edge lists built at level 0,
    certificate tasks after squarings 2 .. S - 1, and a certified level that
    copies D forward instead of squaring.  Sparse random graphs (the
    certificate passes), a dense one (its rows overflow the lists), a
    directed path (it fails until the last squaring), for every size
    (BTAS_BATCH_CERT_MIN_N=0): all equal the oracle and the run without it."""
    import torch
    graphs = []
    for i, n in enumerate((40, 130, 257, 300, 513)):
        graphs.append(gen.random_graph(gen.BASE_SEED, 1700 + i, n, 0.05, 1, 100))
        graphs.append(gen.random_graph(gen.BASE_SEED, 1750 + i, n, min(1.0, 3.0 / n), 1, 10 ** 6))
    graphs.append(gen.random_graph(gen.BASE_SEED, 1790, 300, 0.6, 1, 100))
    P = np.full((150, 150), btas.INF_I32, np.int32)
    np.fill_diagonal(P, 0)
    P[np.arange(149), np.arange(1, 150)] = 4
    graphs.append(P)
    refs = [oracle_mod.floyd_warshall(W) for W in graphs]
    outs = {}
    for name, kv in (("on", {"BTAS_BATCH_CERT_MIN_N": "0"}), ("off", {"BTAS_BATCH_NO_CERT": "1"})):
        os.environ.update(kv)
        try:
            with _tile(tile):
                b = btas.Batch(profile=True)
                Ds = []
                for W in graphs:
                    Wd = dev(W)
                    D = torch.full_like(Wd, -7)
                    b.add_apsp(Wd, D)
                    Ds.append((Wd, D))
                for _ in range(2):
                    b.launch()
                    b.wait()
                outs[name] = [host(D) for _, D in Ds]
                prof = b.profile()
                b.close()
        finally:
            for k in kv:
                del os.environ[k]
        if name == "on":
            assert prof["lists"]["tasks"] > 0 and prof["cert"]["tasks"] > 0
        else:
            assert prof["lists"]["tasks"] == 0 and prof["cert"]["tasks"] == 0
    for W, ref, on, off in zip(graphs, refs, outs["on"], outs["off"]):
        np.testing.assert_array_equal(on, ref, err_msg=f"n={W.shape[0]}")
        np.testing.assert_array_equal(off, ref)


def test_withheld_dependency_times_out(btas):
    """The host withholds one completion of instance 0: its tasks' bounded
    waits run out, the launch reports BTAS_ERR_TIMEOUT, and a later batch on
    the same context still computes correct results."""
    import torch
    import paper_1701_04733_gb300 as b_mod
    W = gen.random_graph(3, 3, 300, 0.1, 1, 100)
    Wd = dev(W)
    D = torch.empty_like(Wd)
    os.environ["BTAS_BATCH_WITHHOLD"] = "0"
    os.environ["BTAS_BATCH_TIMEOUT_CYCLES"] = "2000000"
    try:
        bb = btas.Batch()
        bb.add_apsp(Wd, D)
        bb.launch()
        with pytest.raises(b_mod.BtasError) as ei:
            bb.wait()
        assert ei.value.status == 5
        bb.close()
    finally:
        os.environ.pop("BTAS_BATCH_WITHHOLD", None)
        os.environ.pop("BTAS_BATCH_TIMEOUT_CYCLES", None)
    ok = btas.Batch()
    ok.add_apsp(Wd, D)
    ok.launch()
    ok.wait()
    np.testing.assert_array_equal(host(D), host(btas.apsp(Wd)))
    ok.close()


def test_precision_switches_mid_solve(btas, oracle_mod):
    """Weights near 5000: the first squarings run packed (2*max < 0x7FFF), the
    later ones must fall back to int32 as distances grow; the batch (device
    decision) and the server (host decision) both stay exact, and so does the
    batch with packed squarings disabled."""
    import os
    import torch
    sizes = [40, 130, 257, 300]
    items = []
    for i, n in enumerate(sizes):
        W = gen.random_graph(70 + i, i, n, 0.03, 4000, 5000)
        items.append((W, dev(W), torch.empty((n, n), dtype=torch.int32, device="cuda")))
    for no16, tile in (("0", None), ("1", None), ("0", "64"), ("1", "64")):
        os.environ["BTAS_BATCH_NO_U16"] = no16
        try:
            with _tile(tile):
                b = btas.Batch()
                for _, Wd, D in items:
                    b.add_apsp(Wd, D)
                b.launch()
                b.wait()
                b.close()
        finally:
            os.environ.pop("BTAS_BATCH_NO_U16", None)
        for W, _, D in items:
            np.testing.assert_array_equal(host(D), oracle_mod.floyd_warshall(W), err_msg=f"no16={no16} tile={tile}")
    srv = btas.Server(1 << 30)
    outs = []
    for W, _, _ in items:
        Wh = torch.from_numpy(W).pin_memory()
        Dh = torch.empty_like(Wh).pin_memory()
        srv.submit_apsp(Wh, Dh)
        outs.append((W, Dh))
    srv.wait_all(120)
    srv.close()
    for W, Dh in outs:
        np.testing.assert_array_equal(Dh.numpy(), oracle_mod.floyd_warshall(W))


def test_profile_counts_every_task(btas, oracle_mod):
    """BTAS_BATCH_PROFILE: every task lands in exactly one slot per launch;
    the profiled launch still gives the oracle's results."""
    apsp, gemm = _mixed(btas, seed=3)
    b = btas.Batch(profile=True)
    for W, Wd, D in apsp:
        b.add_apsp(Wd, D)
    for A, B, Ad, Bd, C, sr, tb in gemm:
        b.add_gemm(Ad, Bd, C, sr, trans_b=tb)
    with pytest.raises(btas.BtasError):
        b.profile()  # not launched yet
    for _ in range(2):
        b.launch()
        b.wait()
    prof = b.profile()
    work = {k: v for k, v in prof.items() if k != "wait"}
    assert sum(v["tasks"] for v in work.values()) == 2 * b.tasks
    assert all(v["cycles"] > 0 for v in work.values() if v["tasks"] > 0)
    tiles = lambda x: (x + 127) // 128  # noqa: E731
    n_transposes = sum(tiles(W.shape[0]) ** 2 for W, _, _ in apsp if W.shape[0] > 2) + \
        sum(tiles(A.shape[1]) * tiles(B.shape[1]) for A, B, _, _, _, _, tb in gemm if not tb)
    assert prof["transpose"]["tasks"] == 2 * n_transposes
    assert prof["copy"]["tasks"] == 2 * 2  # n = 1 and n = 2
    assert prof["gemm_i32"]["tasks"] > 0 and prof["gemm_f32"]["tasks"] > 0
    assert prof["apsp_u16"]["tasks"] > 0  # weights <= 100: the packed squaring runs
    assert prof["square_u16"]["tasks"] == prof["square_i32"]["tasks"] == 0
    # graphs of n >= 256 build edge lists and run certificate tasks
    n_lists = 2 * sum((W.shape[0] + 31) // 32 for W, _, _ in apsp if W.shape[0] >= 256)
    assert prof["lists"]["tasks"] == n_lists and prof["cert"]["tasks"] > 0
    for W, Wd, D in apsp:
        np.testing.assert_array_equal(host(D), oracle_mod.apsp_squaring(W))
    for A, B, Ad, Bd, C, sr, tb in gemm:
        np.testing.assert_array_equal(bits(host(C)), bits(oracle_mod.tgemm(sr, A, B)))
    plain = btas.Batch()
    assert btas.btas_batch_profile(plain.handle, None, None, 0) == 1  # created without the flag
    plain.close()
    b.close()


def test_tile_autotuner_table_and_results(btas, oracle_mod):
    """btas_batch_tune times both output tiles per kind and size bucket and
    fills the table; a batch planned afterwards (sizes from several buckets)
    matches the oracle whichever tile each instance took."""
    import torch
    btas.btas_batch_tune_clear()
    assert btas.btas_batch_tile(0, 100) == 0
    res = btas.batch_tune(256)
    for kind in btas.BATCH_TILE_KINDS:
        rows = res[kind]
        assert len(rows) == 8
        for lo, hi, tile, ms128, ms64 in rows:
            assert tile in (64, 128) and ms128 > 0 and ms64 > 0
            assert tile == (64 if ms64 < 0.97 * ms128 else 128)
    assert btas.btas_batch_tile(0, 70) == res["apsp"][2][2]
    apsp, gemm = _mixed(btas, seed=5)
    b = btas.Batch()
    for W, Wd, D in apsp:
        b.add_apsp(Wd, D)
    for A, B, Ad, Bd, C, sr, tb in gemm:
        b.add_gemm(Ad, Bd, C, sr, trans_b=tb)
    b.launch()
    b.wait()
    for W, Wd, D in apsp:
        np.testing.assert_array_equal(host(D), oracle_mod.floyd_warshall(W))
    for A, B, Ad, Bd, C, sr, tb in gemm:
        np.testing.assert_array_equal(bits(host(C)), bits(oracle_mod.tgemm(sr, A, B)))
    # the per-batch choice between the table, all 128 x 128 and all 64 x 64
    mode, ms = b.select_tiles()
    assert mode in ms and ms[mode] == min(ms.values())
    for _, _, D in apsp:
        D.fill_(-5)
    b.launch()
    b.wait()
    for W, Wd, D in apsp:
        np.testing.assert_array_equal(host(D), oracle_mod.floyd_warshall(W))
    b.close()
    btas.btas_batch_tune_clear()
    torch.cuda.synchronize()
