"""GPU parity of APSP by repeated squaring (Sec. III) against the oracle:
Floyd-Warshall (Algorithm 2), the oracle's own squaring, Dijkstra and graph
invariants.  Distances are integers: bit-exact."""
import ctypes
import os

import numpy as np
import pytest

import gen
from gpu_util import INF, dev, host

pytestmark = pytest.mark.gpu


class env:
    """Set environment variables for the duration of a with-block."""

    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        import os
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *a):
        import os
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

PATHS = {"int32": 0x2, "carrier": 0x8, "u16": 0x4}


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def test_config_n256_all_paths(btas, oracle_mod):
    """One random directed graph: n = 256, p = 0.1, w in [1, 100], INF
    off-edges, zero diagonal, 8 squarings; full matrix vs Floyd-Warshall and
    the oracle's squaring."""
    W = gen.random_graph(gen.BASE_SEED, 1, 256, 0.1, 1, 100)
    ref = oracle_mod.floyd_warshall(W)
    np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), ref)
    for name, force in PATHS.items():
        for early in (0, 1):
            D, info = btas.apsp(dev(W), flags=force | early, info=True)
            np.testing.assert_array_equal(host(D), ref, err_msg=f"{name} early={early}")
            # the cooperative kernel may add its sparse first squaring ("sparse")
            reps = set(info["path"].split("+")) - {"sparse"}
            assert reps == {{"int32": "int32", "carrier": "fp32-carrier", "u16": "u16x2"}[name]}
            assert info["bound"] == 255 * int(W[W < INF].max())
    D = host(btas.apsp(dev(W)))
    np.testing.assert_array_equal(D, ref)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 32, 64, 128, 129, 200])
def test_sizes_and_paths(btas, oracle_mod, n):
    """Table II sizes (4..128) plus degenerate and ragged sizes."""
    W = gen.random_graph(gen.BASE_SEED, 200 + n, n, 0.1 if n > 8 else 0.5, 1, 100)
    ref = oracle_mod.floyd_warshall(W)
    for force in PATHS.values():
        np.testing.assert_array_equal(host(btas.apsp(dev(W), flags=force | 1)), ref)


def test_in_place_and_squarings_count(btas, oracle_mod):
    for n in (6, 9, 100, 257):  # odd and even squaring counts
        W = gen.random_graph(3, n, n, 0.05, 0, 50)
        ref = oracle_mod.floyd_warshall(W)
        for force in PATHS.values():
            t = dev(W)
            D, info = btas.apsp(t, out=t, flags=force | 1, info=True)
            np.testing.assert_array_equal(host(t), ref)
            assert 0 <= info["squarings"] <= btas.btas_apsp_squarings(n)


def test_chain_uses_every_squaring(btas):
    """A directed path needs all ceil(log2(n-1)) squarings: early exit must
    not stop it, and the count of changing squarings equals S."""
    n = 300
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 1
    D, info = btas.apsp(dev(W), flags=0x1 | 0x2, info=True)
    D = host(D)
    assert D[0, n - 1] == n - 1 and D[n - 1, 0] == INF
    assert info["squarings"] == btas.btas_apsp_squarings(n)


def test_early_exit_converges(btas, oracle_mod):
    """A dense graph has shortest paths of few edges: early exit stops after a
    couple of squarings and gives the same matrix."""
    W = gen.random_graph(4, 4, 500, 0.5, 1, 10)
    ref = oracle_mod.floyd_warshall(W)
    D, info = btas.apsp(dev(W), flags=0x1 | 0x2, info=True)
    np.testing.assert_array_equal(host(D), ref)
    assert info["squarings"] < btas.btas_apsp_squarings(500)


def test_domain_errors(btas):
    import paper_1701_04733_gb300 as b
    W = gen.random_graph(5, 5, 40, 0.2, 1, 9)
    bad = W.copy()
    bad[0, 1] = -3
    with pytest.raises(b.BtasError):
        btas.apsp(dev(bad))
    bad = W.copy()
    bad[2, 2] = 4
    with pytest.raises(b.BtasError):
        btas.apsp(dev(bad))
    big = W.copy()
    big[0, 1] = 10 ** 6  # bound 39e6 > 2^23 and > 0x7FFF
    with pytest.raises(b.BtasError):
        btas.apsp(dev(big), flags=0x4 | 1)
    with pytest.raises(b.BtasError):
        btas.apsp(dev(big), flags=0x8 | 1)


def test_u16_entry_point(btas, oracle_mod):
    import torch
    n = 300
    W32 = gen.random_graph(6, 6, n, 0.05, 1, 7)
    W16 = np.where(W32 == INF, 0x7FFF, W32).astype(np.uint16)
    ref = oracle_mod.apsp_squaring(W16)
    D = btas.apsp_u16(dev(W16.view(np.int16)), 7)
    np.testing.assert_array_equal(host(D).view(np.uint16), ref)
    t = dev(W16.view(np.int16))
    btas.apsp_u16(t, 7, out=t, early_exit=False)
    np.testing.assert_array_equal(host(t).view(np.uint16), ref)


def test_config_n4096_packed_vs_int32(btas, oracle_mod):
    """n = 4096, p = 0.05, w in [1, 7]: (n-1)*7 = 28665 < 0x7FFF.  The packed
    16-bit path and the int32 path agree bit-exactly, and 64 seeded rows
    match Dijkstra."""
    n = 4096
    W = gen.random_graph(gen.BASE_SEED, 3, n, 0.05, 1, 7)
    Wd = dev(W)
    D16, i16 = btas.apsp(Wd, flags=0x4 | 1, info=True)
    D32, i32 = btas.apsp(Wd, flags=0x2 | 1, info=True)
    assert i16["bound"] == (n - 1) * 7
    D16, D32 = host(D16), host(D32)
    np.testing.assert_array_equal(D16, D32)
    srcs = gen.sample_indices(gen.BASE_SEED, 33, 64, n)
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        rows = oracle_mod.dijkstra_rows(W, srcs)
    finally:
        oracle_mod.set_threads(1)
    np.testing.assert_array_equal(D16[srcs], rows)


def test_config_n8192_sampled(btas, oracle_mod):
    """n = 8192, p = 0.01, w in [1, 1000], 13 squarings: 64 seeded Dijkstra
    rows, plus the fixpoint D (x) D = D on 64 seeded rows (oracle product
    rows) and the zero diagonal."""
    n = 8192
    W = gen.random_graph(gen.BASE_SEED, 2, n, 0.01, 1, 1000)
    D, info = btas.apsp(dev(W), info=True)
    D = host(D)
    assert (np.diag(D) == 0).all()
    srcs = gen.sample_indices(gen.BASE_SEED, 34, 64, n)
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        np.testing.assert_array_equal(D[srcs], oracle_mod.dijkstra_rows(W, srcs))
        np.testing.assert_array_equal(oracle_mod.tgemm(0, D[srcs], D), D[srcs])
    finally:
        oracle_mod.set_threads(1)
    # the int32 kernels agree with the automatically chosen path
    D32 = host(btas.apsp(dev(W), flags=0x2 | 1))
    np.testing.assert_array_equal(D32, D)


def test_workspace_pool_caches_and_trims(btas, oracle_mod):
    """The tiled path's workspace comes from the library's pool: it stays
    reserved between calls (later calls reuse it) and btas_workspace_trim
    releases it.  The cooperative path's small workspaces come from a cache
    of the calling thread instead: repeated calls take nothing from the
    pool."""
    W = gen.random_graph(91, 1, 300, 0.05, 1, 100)
    with env(BTAS_APSP_NO_MID="1"):
        D1 = host(btas.apsp(dev(W)))
        held = btas.btas_workspace_reserved()
        assert held > 0
        D2 = host(btas.apsp(dev(W)))
        assert btas.btas_workspace_reserved() == held
    np.testing.assert_array_equal(D1, D2)
    np.testing.assert_array_equal(D1, oracle_mod.apsp_squaring(W))
    assert btas.btas_workspace_trim() == 0
    assert btas.btas_workspace_reserved() < held
    before = btas.btas_workspace_reserved()
    for _ in range(3):
        np.testing.assert_array_equal(host(btas.apsp(dev(W))), D1)  # cooperative kernel
    assert btas.btas_workspace_reserved() == before


@pytest.fixture
def one_block_up_to_128():
    """Send every n <= 128 to the one-block kernel (by default only the
    smallest graphs take it, the rest the cooperative kernel)."""
    with env(BTAS_APSP_SMALL_MAX_N="128"):
        yield


@pytest.mark.parametrize("n", [3, 4, 7, 33, 64, 100, 127, 128])
def test_small_graph_single_block_path(btas, oracle_mod, n, one_block_up_to_128):
    """n <= 128 runs in one thread block (all squarings in shared memory);
    distances, squarings count and bound equal the general path's and the
    oracle's, with and without early exit, in place too."""
    import os
    for p, whi in ((0.5 if n < 8 else 0.1, 100), (0.03, 10 ** 6)):
        W = gen.random_graph(gen.BASE_SEED, 700 + n, n, p, 1, whi)
        ref = oracle_mod.floyd_warshall(W)
        for early in (0, 1):
            D, info = btas.apsp(dev(W), flags=early, info=True)
            os.environ["BTAS_APSP_NO_SMALL"] = "1"
            try:
                D2, info2 = btas.apsp(dev(W), flags=early | btas.APSP_FORCE_I32, info=True)
            finally:
                del os.environ["BTAS_APSP_NO_SMALL"]
            np.testing.assert_array_equal(host(D), ref)
            np.testing.assert_array_equal(host(D2), ref)
            assert info["path"] == "int32"
            assert info["squarings"] == info2["squarings"]
            assert info["bound"] == info2["bound"] == (n - 1) * int(W[W < INF].max())
        t = dev(W)
        btas.apsp(t, out=t)
        np.testing.assert_array_equal(host(t), ref)
    # a directed path needs every squaring
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 3
    D, info = btas.apsp(dev(W), info=True)
    assert host(D)[0, n - 1] == 3 * (n - 1)
    assert info["squarings"] == btas.btas_apsp_squarings(n)
    # domain violations are reported and leave D untouched
    bad = W.copy()
    bad[1, 1] = 7
    out = dev(np.full((n, n), 123, np.int32))
    with pytest.raises(btas.BtasError):
        btas.apsp(dev(bad), out=out)
    assert (host(out) == 123).all()


@pytest.fixture
def cooperative_from_3():
    """Send every n >= 3 up to the cooperative kernel's limit to it, with its
    edge lists at every size (by default from n = 384)."""
    with env(BTAS_APSP_SMALL_MAX_N="0", BTAS_MID_LISTS_MIN_N="0"):
        yield


@pytest.mark.parametrize("n", [3, 7, 33, 100, 129, 200, 256, 333, 512, 777, 1024])
def test_mid_graph_cooperative_path(btas, oracle_mod, n, cooperative_from_3):
    """Up to n = 1024 every squaring can run in one cooperative launch (split-k
    pieces merged with atomicMin, one grid barrier per squaring), each
    squaring on packed 16-bit pairs while the largest merged value allows it
    (<= 16383), else on int32.  Distances, squarings count and bound equal the
    general path's and the oracle's, with and without early exit, with the
    packed squarings disabled (BTAS_MID_NO_U16=1, FORCE_I32), and in place."""
    for p, whi, expect in ((0.05, 100, "u16x2"), (3.0 / n, 10 ** 6, "int32"), (0.02, 12000, None)):
        W = gen.random_graph(gen.BASE_SEED, 800 + n, n, p, 1, whi)
        ref = oracle_mod.floyd_warshall(W)
        for early in (0, 1):
            D, info = btas.apsp(dev(W), flags=early, info=True)
            with env(BTAS_APSP_NO_MID="1"):
                D2, info2 = btas.apsp(dev(W), flags=early | btas.APSP_FORCE_I32, info=True)
            with env(BTAS_MID_NO_U16="1"):
                D3, info3 = btas.apsp(dev(W), flags=early, info=True)
            D4, info4 = btas.apsp(dev(W), flags=early | btas.APSP_FORCE_I32, info=True)
            with env(BTAS_MID_NO_SPARSE="1", BTAS_MID_NO_CERT="1"):  # every squaring dense, none skipped
                D5, info5 = btas.apsp(dev(W), flags=early, info=True)
            for X in (D, D2, D3, D4, D5):
                np.testing.assert_array_equal(host(X), ref)
            # these graphs have few edges per row: the first squaring runs on the edge lists
            assert "sparse" in info["path"].split("+")
            if expect is None:  # first squaring packed (max w <= 16383), later ones on int32
                assert "u16x2" in info5["path"].split("+")
            else:
                assert info5["path"] == expect
                assert set(info["path"].split("+")) - {"sparse"} <= {expect}
            assert set(info3["path"].split("+")) - {"sparse"} <= {"int32"}
            assert set(info4["path"].split("+")) - {"sparse"} <= {"int32"}
            assert info5["path"] != "" and "sparse" not in info5["path"]
            assert (info["squarings"] == info2["squarings"] == info3["squarings"] == info4["squarings"]
                    == info5["squarings"])
            assert info["bound"] == info2["bound"] == info5["bound"] == (n - 1) * int(W[W < INF].max())
        t = dev(W)
        btas.apsp(t, out=t)
        np.testing.assert_array_equal(host(t), ref)
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 5
    D, info = btas.apsp(dev(W), info=True)
    assert host(D)[0, n - 1] == 5 * (n - 1)
    assert info["squarings"] == btas.btas_apsp_squarings(n)
    bad = W.copy()
    bad[1, n - 1] = -1
    out = dev(np.full((n, n), 77, np.int32))
    with pytest.raises(btas.BtasError):
        btas.apsp(dev(bad), out=out)
    assert (host(out) == 77).all()


def test_cooperative_path_above_1024(btas, oracle_mod):
    """The cooperative kernel serves btas_apsp up to n = 1792 by default; at
    n = 1536 it equals the oracle and counts the tiled path's squarings."""
    n = 1536
    W = gen.random_graph(gen.BASE_SEED, 950, n, 0.02, 1, 100)
    ref = oracle_mod.floyd_warshall(W)
    D, info = btas.apsp(dev(W), info=True)
    with env(BTAS_APSP_NO_MID="1"):
        _, info2 = btas.apsp(dev(W), flags=btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32, info=True)
    np.testing.assert_array_equal(host(D), ref)
    assert info["path"] == "u16x2+sparse"  # the first squaring from the edge lists
    assert info["squarings"] == info2["squarings"]


@pytest.mark.parametrize("wide", ["0", "1"])
def test_cooperative_barrier_timeout_is_reported(btas, oracle_mod, wide):
    """Failure detection without a fault: with BTAS_MID_WITHHOLD=1 one block of
    the cooperative kernel (64 x 64 form, or the warp-specialised 128 x 128
    form) never arrives at its first grid barrier, the others' bounded waits
    expire (about 2 s), and the call returns BTAS_ERR_TIMEOUT with D
    untouched; the next call on the same context succeeds."""
    import torch
    n = 300
    W = gen.random_graph(gen.BASE_SEED, 960, n, 0.05, 1, 100)
    out = dev(np.full((n, n), 41, np.int32))
    with env(BTAS_MID_WIDE_MIN_N="0" if wide == "1" else "100000"):
        with env(BTAS_MID_WITHHOLD="1"):
            with pytest.raises(btas.BtasError) as ei:
                btas.apsp(dev(W), out=out)
        assert ei.value.status == 5
        assert (host(out) == 41).all()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(btas.apsp(dev(W))), oracle_mod.floyd_warshall(W))


@pytest.mark.parametrize("n", [3, 7, 129, 200, 333, 513, 1100])
def test_wide_cooperative_form(btas, oracle_mod, n, cooperative_from_3):
    """The warp-specialised 128 x 128 form of the cooperative kernel (producer
    warps staging through an mbarrier ring, consumer warps with 8 x 8
    outputs), forced at every size with BTAS_MID_WIDE_MIN_N=0: ragged edges of
    the 128-wide tiles, packed and int32 squarings, early exit or not, in
    place.  Same distances and squarings count as the oracle and the tiled
    path."""
    with env(BTAS_MID_WIDE_MIN_N="0"):
        for p, whi in ((0.05, 100), (3.0 / n, 10 ** 6), (0.02, 12000)):
            W = gen.random_graph(gen.BASE_SEED, 980 + n, n, p, 1, whi)
            ref = oracle_mod.floyd_warshall(W)
            for early in (0, 1):
                D, info = btas.apsp(dev(W), flags=early, info=True)
                with env(BTAS_APSP_NO_MID="1"):
                    _, info2 = btas.apsp(dev(W), flags=early | btas.APSP_FORCE_I32, info=True)
                np.testing.assert_array_equal(host(D), ref)
                assert info["squarings"] == info2["squarings"]
            t = dev(W)
            btas.apsp(t, out=t)
            np.testing.assert_array_equal(host(t), ref)


def _cap(n):
    """Edges per row the cooperative kernel's lists hold by default."""
    return min(256, max(32, ((n // 4 + 31) // 32) * 32))


def _graphs_for_lists(n):
    """Graphs for the edge-list paths: sparse random graphs (the usual
    case), a dense one (its rows overflow the lists, so every squaring is
    dense), a directed path (every squaring lowers entries, so a certificate
    tried after each one fails until the last), and rows with exactly cap and
    cap + 1 edges."""
    out = [("p0.05", gen.random_graph(gen.BASE_SEED, 1200 + n, n, 0.05, 1, 100)),
           ("p3/n", gen.random_graph(gen.BASE_SEED, 1300 + n, n, min(1.0, 3.0 / n), 1, 10 ** 6)),
           ("dense", gen.random_graph(gen.BASE_SEED, 1400 + n, n, 0.6, 1, 1000))]
    P = np.full((n, n), INF, np.int32)
    np.fill_diagonal(P, 0)
    P[np.arange(n - 1), np.arange(1, n)] = 7
    out.append(("path", P))
    cap = _cap(n)
    if cap + 2 <= n:
        for extra in (0, 1):
            G = gen.random_graph(gen.BASE_SEED, 1500 + n + extra, n, 2.0 / n, 1, 50)
            row = G[1].copy()
            row[:] = INF
            row[1] = 0
            cols = [j for j in range(n) if j != 1][: cap + extra]
            row[cols] = np.arange(1, len(cols) + 1, dtype=np.int32) % 97 + 1
            G[1] = row
            out.append((f"deg{cap + extra}", G))
    return out


@pytest.mark.parametrize("wide", [False, True])
@pytest.mark.parametrize("n", [65, 130, 257, 700, 1100])
def test_edge_lists_and_certificate(btas, oracle_mod, n, wide, cooperative_from_3):
    """The cooperative kernel's edge lists: the first squaring as sparse
    products over them (rows with at most cap edges), and the closure
    certificate that stops a solve without the squaring that would only
    confirm the fixpoint.  Every setting -- both on (default), the certificate
    tried after every changing squaring (BTAS_MID_CERT_ALWAYS=1), lists too
    short for any row (BTAS_MID_LIST_CAP=4), either one off -- gives the
    oracle's distances and the squarings count and bound of the run with
    both off, in both forms of the kernel, with and without early exit."""
    settings = ({}, {"BTAS_MID_CERT_ALWAYS": "1"}, {"BTAS_MID_LIST_CAP": "4"}, {"BTAS_MID_NO_SPARSE": "1"},
                {"BTAS_MID_NO_CERT": "1"})
    form = {"BTAS_MID_WIDE_MIN_N": "0" if wide else "100000"}
    for name, W in _graphs_for_lists(n):
        ref = oracle_mod.floyd_warshall(W)
        deg = ((W < INF).sum(1) - 1).max()
        for early in (0, 1):
            with env(BTAS_MID_NO_SPARSE="1", BTAS_MID_NO_CERT="1", **form):
                D0, info0 = btas.apsp(dev(W), flags=early, info=True)
            np.testing.assert_array_equal(host(D0), ref)
            for extra in settings:
                with env(**form, **extra):
                    D, info = btas.apsp(dev(W), flags=early, info=True)
                np.testing.assert_array_equal(host(D), ref, err_msg=f"{name} {extra} early={early}")
                assert info["squarings"] == info0["squarings"], (name, extra, early)
                assert info["bound"] == info0["bound"]
                lists_hold = deg <= int(extra.get("BTAS_MID_LIST_CAP", _cap(n)))
                used = "sparse" in info["path"].split("+")
                assert used == (lists_hold and "BTAS_MID_NO_SPARSE" not in extra), (name, extra, info["path"])
        t = dev(W)
        btas.apsp(t, out=t)
        np.testing.assert_array_equal(host(t), ref)


@pytest.mark.parametrize("n,lists", [(256, False), (383, False), (384, True), (512, True)])
def test_edge_lists_size_floor(btas, oracle_mod, n, lists):
    """By default the cooperative kernel builds its edge lists from n = 384:
    below it a squaring is bound by the grid barrier and the shortcuts do not
    pay.  Distances equal the oracle's either way."""
    W = gen.random_graph(gen.BASE_SEED, 1650 + n, n, 0.05, 1, 100)
    D, info = btas.apsp(dev(W), info=True)
    np.testing.assert_array_equal(host(D), oracle_mod.floyd_warshall(W))
    assert ("sparse" in info["path"].split("+")) == lists, info["path"]


def test_edge_lists_allocation_free(btas, oracle_mod, cooperative_from_3):
    """The allocation-free entry point gives the cooperative kernel room for
    its edge lists up to n = 1024: same distances and squarings as
    btas_apsp."""
    import torch
    for n in (300, 1024):
        W = gen.random_graph(gen.BASE_SEED, 1600 + n, n, 0.05, 1, 100)
        ref = oracle_mod.floyd_warshall(W)
        Wd = dev(W)
        D = torch.empty_like(Wd)
        st = torch.cuda.current_stream().cuda_stream
        assert btas.btas_apsp_noalloc(n, Wd.data_ptr(), D.data_ptr(), st) == 0
        sq = ctypes.c_int(-1)
        assert btas.btas_apsp_noalloc_status(st, ctypes.addressof(sq)) == 0
        np.testing.assert_array_equal(host(D), ref)
        _, info = btas.apsp(Wd, info=True)
        assert sq.value == info["squarings"]


@pytest.mark.parametrize("n", [2304, 2560, 3000])
def test_cooperative_above_1792_for_sparse_graphs(btas, oracle_mod, n):
    """Above n = 1792 btas_apsp keeps a graph on the cooperative kernel when
    every row fits its edge lists (p = 0.02 here): distances equal
    Floyd-Warshall's and the squarings count equals the tiled path's."""
    W = gen.random_graph(gen.BASE_SEED, 990 + n, n, 0.02, 1, 100)
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle_mod.floyd_warshall(W)
    finally:
        oracle_mod.set_threads(1)
    D, info = btas.apsp(dev(W), info=True)
    with env(BTAS_APSP_NO_MID="1"):
        D2, info2 = btas.apsp(dev(W), info=True)
    np.testing.assert_array_equal(host(D), ref)
    np.testing.assert_array_equal(host(D2), ref)
    assert info["squarings"] == info2["squarings"]
    assert "sparse" in info["path"].split("+") and "sparse" not in info2["path"]


def test_dense_graph_above_1792_goes_tiled(btas, oracle_mod):
    """A graph too dense for the edge lists (p = 0.5 at n = 2048) is declined
    by the cooperative kernel after its domain check and solved on the tiled
    kernels: same distances as Floyd-Warshall, and a domain error is still
    reported with D untouched."""
    n = 2048
    W = gen.random_graph(gen.BASE_SEED, 995, n, 0.5, 1, 1000)
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle_mod.floyd_warshall(W)
    finally:
        oracle_mod.set_threads(1)
    D, info = btas.apsp(dev(W), info=True)
    np.testing.assert_array_equal(host(D), ref)
    assert "sparse" not in info["path"]
    bad = W.copy()
    bad[5, 5] = 3
    out = dev(np.full((n, n), 11, np.int32))
    with pytest.raises(btas.BtasError):
        btas.apsp(dev(bad), out=out)
    assert (host(out) == 11).all()
