"""Pins for the oracle's APSP routines: repeated squaring (Sec. III),
Floyd-Warshall (Algorithm 2), Dijkstra and brute force.  They are checked
against a hand-worked graph, against each other (four different algorithms
reaching one unique distance matrix), and against graph invariants."""
import itertools
from collections import deque

import numpy as np
import pytest

import gen
from golden import as_f32, as_i32, load

INF = 0x3FFFFFFF


def _bfs_reach(W):
    n = W.shape[0]
    R = np.zeros((n, n), bool)
    for s in range(n):
        seen = {s}
        q = deque([s])
        while q:
            u = q.popleft()
            for v in range(n):
                if W[u, v] != INF and v not in seen:
                    seen.add(v)
                    q.append(v)
        R[s, list(seen)] = True
    return R


def _check_invariants(oracle_mod, W, D):
    n = W.shape[0]
    assert (np.diag(D) == 0).all()
    assert (D <= W).all()
    # INF pattern = complement of reachability (BFS, no weights involved)
    np.testing.assert_array_equal(D != INF, _bfs_reach(W))
    # triangle inequality over finite entries
    Dl = np.where(D == INF, 1 << 40, D.astype(np.int64))
    via = (Dl[:, :, None] + Dl[None, :, :]).min(axis=1)
    assert (Dl <= via).all()
    # fixpoint of the squaring: D (x) D == D
    np.testing.assert_array_equal(oracle_mod.tgemm(0, D, D), D)


def test_squarings_closed_form(oracle_mod):
    expect = {0: 0, 1: 0, 2: 0, 3: 1, 4: 2, 5: 2, 6: 3, 9: 3, 10: 4, 17: 4, 18: 5,
              256: 8, 257: 8, 258: 9, 1024: 10, 4096: 12, 8192: 13}
    for n, s in expect.items():
        assert oracle_mod.apsp_squarings(n) == s, n
        if n >= 3:
            assert 2 ** s >= n - 1 > 2 ** (s - 1) if s > 0 else n - 1 <= 1


def test_hand_worked_graph(oracle_mod):
    g = load("apsp_6node.txt")
    W, D = as_i32(g["W"]), as_i32(g["D"])
    np.testing.assert_array_equal(oracle_mod.floyd_warshall(W), D)
    np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), D)
    np.testing.assert_array_equal(oracle_mod.bruteforce_apsp(W), D)
    np.testing.assert_array_equal(oracle_mod.dijkstra_rows(W, np.arange(6)), D)
    # d(1,2) = 12 uses the 4-edge path 1->3->4->0->2: one squaring (walks of
    # <= 2 edges) cannot see it, two squarings (<= 4 edges) can.  d(5,4) = 9
    # uses the 5-edge path 5->0->2->1->3->4 and needs the third squaring; the
    # best walk of <= 4 edges is 5->0->1->3->4 = 10.
    D1 = oracle_mod.apsp_squaring(W, 1)
    D2 = oracle_mod.apsp_squaring(W, 2)
    assert D1[1, 2] == INF and D2[1, 2] == 12 == D[1, 2]
    assert D2[5, 4] == 10 and D[5, 4] == 9
    diff = np.argwhere(D2 != D)
    np.testing.assert_array_equal(diff, [[5, 4]])


def test_all_three_vertex_graphs(oracle_mod):
    """Every directed graph on 3 vertices (2^6 edge sets), weights 1..9."""
    offd = [(i, j) for i in range(3) for j in range(3) if i != j]
    for mask in range(1 << 6):
        W = np.full((3, 3), INF, np.int32)
        np.fill_diagonal(W, 0)
        for b, (i, j) in enumerate(offd):
            if mask >> b & 1:
                W[i, j] = 1 + (mask * 7 + b * 5) % 9
        D = oracle_mod.bruteforce_apsp(W)
        np.testing.assert_array_equal(oracle_mod.floyd_warshall(W), D)
        np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), D)


@pytest.mark.parametrize("n", [2, 4, 5, 6, 7, 8])
def test_random_small_vs_bruteforce(oracle_mod, n):
    for seed in range(25):
        W = gen.random_graph(seed, n, n, 0.45, 0, 20)
        D = oracle_mod.bruteforce_apsp(W)
        np.testing.assert_array_equal(oracle_mod.floyd_warshall(W), D)
        np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), D)
        np.testing.assert_array_equal(oracle_mod.dijkstra_rows(W, np.arange(n)), D)


@pytest.mark.parametrize("n", [4, 16, 32, 64, 128])
def test_paper_sizes_fw_squaring_dijkstra(oracle_mod, n):
    """The random-matrix sizes of Table II (4..128 vertices)."""
    W = gen.random_graph(gen.BASE_SEED, 100 + n, n, 0.1, 1, 100)
    D = oracle_mod.floyd_warshall(W)
    np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), D)
    np.testing.assert_array_equal(oracle_mod.dijkstra_rows(W, np.arange(n)), D)
    _check_invariants(oracle_mod, W, D)


def test_config_graph_n256(oracle_mod):
    """One random directed graph, n = 256, p = 0.1, w in [1, 100], 8 squarings."""
    W = gen.random_graph(gen.BASE_SEED, 1, 256, 0.1, 1, 100)
    oracle_mod.set_threads(4)
    try:
        D = oracle_mod.apsp_squaring(W)
        np.testing.assert_array_equal(oracle_mod.floyd_warshall(W), D)
        np.testing.assert_array_equal(oracle_mod.dijkstra_rows(W, [0, 17, 255]), D[[0, 17, 255]])
        _check_invariants(oracle_mod, W, D)
    finally:
        oracle_mod.set_threads(1)


def test_zero_weight_edges_and_disconnected(oracle_mod):
    W = gen.random_graph(5, 5, 40, 0.05, 0, 3)
    D = oracle_mod.floyd_warshall(W)
    np.testing.assert_array_equal(oracle_mod.apsp_squaring(W), D)
    _check_invariants(oracle_mod, W, D)
    assert (D == INF).any()


def test_u16_squaring_matches_int32_under_bound(oracle_mod):
    """n = 64, w in [1, 7]: (n-1)*7 = 441 < 0x7FFF, so the 16-bit squaring is
    exact and equals the int32 one with INF16 widened to INF."""
    W32 = gen.random_graph(7, 3, 64, 0.05, 1, 7)
    W16 = np.where(W32 == INF, 0x7FFF, W32).astype(np.uint16)
    D16 = oracle_mod.apsp_squaring(W16).astype(np.int64)
    D32 = oracle_mod.apsp_squaring(W32)
    np.testing.assert_array_equal(np.where(D16 == 0x7FFF, INF, D16), D32)


def test_chain_needs_all_squarings(oracle_mod):
    """A directed path 0->1->...->n-1 has a shortest path of n-1 edges, so it
    needs exactly ceil(log2(n-1)) squarings."""
    n = 9
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    for i in range(n - 1):
        W[i, i + 1] = 1
    S = oracle_mod.apsp_squarings(n)
    D = oracle_mod.apsp_squaring(W, S)
    assert D[0, n - 1] == n - 1
    assert oracle_mod.apsp_squaring(W, S - 1)[0, n - 1] == INF
    for i, j in itertools.product(range(n), range(n)):
        assert D[i, j] == (j - i if j >= i else INF)


def _walk(W, Nx, i, j):
    """Follow the next-hop matrix from i to j; returns the walk's weight."""
    total, v, steps = 0, i, 0
    while v != j:
        u = int(Nx[v, j])
        assert u >= 0 and W[v, u] != INF, (i, j, v, u)
        total += int(W[v, u])
        v = u
        steps += 1
        assert steps <= W.shape[0], "next-hop walk does not terminate"
    return total


def test_paths_hand_worked(oracle_mod):
    g = load("apsp_paths_5node.txt")
    W, D, N = as_i32(g["W"]), as_i32(g["D"]), as_i32(g["N"])
    d, nx = oracle_mod.apsp_paths(W)
    np.testing.assert_array_equal(d, D)
    np.testing.assert_array_equal(nx, N)
    np.testing.assert_array_equal(d, oracle_mod.floyd_warshall(W))


@pytest.mark.parametrize("n", [3, 8, 40, 100])
def test_paths_are_valid_shortest_walks(oracle_mod, n):
    """Following Next from i reaches j with total weight D[i][j] (positive
    weights), Next is -1 exactly where D is INF, and D equals Floyd-Warshall."""
    W = gen.random_graph(11, n, n, 0.15 if n > 8 else 0.5, 1, 30)
    D, Nx = oracle_mod.apsp_paths(W)
    np.testing.assert_array_equal(D, oracle_mod.floyd_warshall(W))
    assert ((Nx == -1) == (D == INF)).all()
    for i in range(n):
        for j in range(n):
            if D[i, j] != INF:
                assert _walk(W, Nx, i, j) == D[i, j]


def _as_float_graph(W):
    """An int32 graph as binary32 weights (INF -> +inf); exact for the small
    integer weights used here."""
    return np.where(W == INF, np.float32(np.inf), W.astype(np.float32)).astype(np.float32)


def test_paths_f32_rounding_tie(oracle_mod):
    """A hand-worked binary32 case whose tie exists only after rounding: the
    smallest minimising k keeps the direct edge."""
    g = load("apsp_paths_f32_rounding_3node.txt")
    W, D, N = as_f32(g["W"]), as_f32(g["D"]), as_i32(g["N"])
    d, nx = oracle_mod.apsp_paths(W)
    np.testing.assert_array_equal(d.view(np.uint32), D.view(np.uint32))
    np.testing.assert_array_equal(nx, N)


@pytest.mark.parametrize("n", [3, 8, 40])
def test_paths_f32_equal_int32_on_integer_weights(oracle_mod, n):
    """Integer weights whose path sums stay below 2^24 are exact in binary32:
    the fp32 next-hop squaring then gives the int32 routine's distances and
    next hops, ties included (weights 1..6 make many)."""
    W = gen.random_graph(21, n, n, 0.3 if n > 8 else 0.6, 1, 6)
    d32, n32 = oracle_mod.apsp_paths(W)
    df, nf = oracle_mod.apsp_paths(_as_float_graph(W))
    np.testing.assert_array_equal(df, _as_float_graph(d32))
    np.testing.assert_array_equal(nf, n32)


@pytest.mark.parametrize("n", [5, 30])
def test_paths_f32_distances_are_repeated_products(oracle_mod, n):
    """With rounding in play (weights U[0,1)), the distances are those of the
    same number of squarings by the tropical product routine, bit for bit,
    and the next hop is -1 exactly where the distance is +inf."""
    W = _as_float_graph(gen.random_graph(22, n, n, 0.4, 1, 2)).copy()
    u = gen.uniform_f32(23, n, (n, n))
    W = np.where(np.isinf(W) | (np.eye(n) == 1), W, u).astype(np.float32)
    S = oracle_mod.apsp_squarings(n)
    d, nx = oracle_mod.apsp_paths(W)
    ref = W.copy()
    for _ in range(S):
        ref = oracle_mod.tgemm(0, ref, ref)
    np.testing.assert_array_equal(d.view(np.uint32), ref.view(np.uint32))
    assert ((nx == -1) == np.isinf(d)).all()
