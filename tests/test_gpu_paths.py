"""APSP with path reconstruction: distances and the next-hop matrix are
bit-identical to the oracle's squaring with the smallest-minimising-k rule,
and every next-hop walk is a shortest path."""
import numpy as np
import pytest

import gen
from golden import as_f32, as_i32, load
from gpu_util import INF, bits, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def test_hand_worked(btas):
    g = load("apsp_paths_5node.txt")
    D, Nx = btas.apsp_paths(dev(as_i32(g["W"])))
    np.testing.assert_array_equal(host(D), as_i32(g["D"]))
    np.testing.assert_array_equal(host(Nx), as_i32(g["N"]))


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


@pytest.mark.parametrize("keyed", ["1", "0"])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 64, 65, 200, 513])
def test_matches_oracle_and_walks_are_shortest(btas, oracle_mod, n, keyed):
    """Weights 1..20, so equal-length alternatives are common and the
    smallest-k rule decides many next hops.  keyed = 1: each squaring is one
    int32 product of (value << 13 | k) keys; keyed = 0
    (BTAS_PATHS_NO_KEYED=1): the argmin kernel."""
    W = gen.random_graph(21, n, n, 0.08 if n > 10 else 0.5, 1, 20)
    ref_d, ref_n = oracle_mod.apsp_paths(W)
    for early in (True, False):
        with env(BTAS_PATHS_NO_KEYED="0" if keyed == "1" else "1"):
            D, Nx = btas.apsp_paths(dev(W), early_exit=early)
        np.testing.assert_array_equal(host(D), ref_d)
        np.testing.assert_array_equal(host(Nx), ref_n)
    D, Nx = host(D), host(Nx)
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j = (int(x) for x in rng.integers(0, n, 2))
        if D[i, j] == INF:
            assert Nx[i, j] == -1
            continue
        v, tot, steps = i, 0, 0
        while v != j:
            u = int(Nx[v, j])
            tot += int(W[v, u])
            v = u
            steps += 1
            assert steps <= n
        assert tot == D[i, j]


@pytest.mark.parametrize("whi", [30000, 10 ** 6])
def test_large_weights(btas, oracle_mod, whi):
    """Weights up to 30000: the first squaring is keyed (every entry <=
    49151), later ones, whose sums may exceed the key range, run on the
    argmin kernel; weights up to 10^6: the argmin kernel throughout.  Same
    bits as the oracle either way, with ties among the 10^6 weights made by
    repeated weights."""
    n = 300
    W = gen.random_graph(22, whi % 97, n, 0.05, 1, whi)
    W[(W != INF) & (W > 0)] = (W[(W != INF) & (W > 0)] // 7) * 7 + 7  # coarser weights: more ties
    np.fill_diagonal(W, 0)
    ref_d, ref_n = oracle_mod.apsp_paths(W)
    D, Nx = btas.apsp_paths(dev(W))
    np.testing.assert_array_equal(host(D), ref_d)
    np.testing.assert_array_equal(host(Nx), ref_n)


def _f32_graph(seed, n, p, integer_weights):
    """A binary32 graph: +inf for no edge, zero diagonal; weights U[0, 1) or
    small integers (many ties)."""
    W = gen.random_graph(seed, n, n, p, 1, 6).astype(np.float32)
    W[W == np.float32(INF)] = np.float32(np.inf)
    if not integer_weights:
        u = gen.uniform_f32(seed + 1, n, (n, n))
        W = np.where(np.isinf(W) | (np.eye(n) == 1), W, u).astype(np.float32)
    return W


def test_f32_hand_worked_rounding_tie(btas):
    """The binary32 fixture whose tie only the rounding creates."""
    g = load("apsp_paths_f32_rounding_3node.txt")
    D, Nx = btas.apsp_paths(dev(as_f32(g["W"])))
    np.testing.assert_array_equal(host(D).view(np.uint32), as_f32(g["D"]).view(np.uint32))
    np.testing.assert_array_equal(host(Nx), as_i32(g["N"]))


@pytest.mark.parametrize("integer_weights", [False, True])
@pytest.mark.parametrize("n", [2, 5, 63, 64, 65, 130, 300])
def test_f32_matches_oracle(btas, oracle_mod, n, integer_weights):
    """Distances bit for bit and next hops equal to the oracle's binary32
    squaring, over ragged sizes around the 64-wide tile, with rounding in
    play (weights U[0, 1)) and with many ties (integer weights)."""
    W = _f32_graph(400 + n, n, 0.2 if n > 8 else 0.6, integer_weights)
    D, Nx = btas.apsp_paths(dev(W))
    d_ref, n_ref = oracle_mod.apsp_paths(W)
    np.testing.assert_array_equal(host(D).view(np.uint32), d_ref.view(np.uint32))
    np.testing.assert_array_equal(host(Nx), n_ref)


def test_f32_domain_is_checked(btas):
    """NaN, a negative weight or a non-zero diagonal entry: BTAS_ERR_ARG,
    nothing written."""
    import torch
    base = _f32_graph(410, 40, 0.2, False)
    for r, c, v in ((3, 4, np.float32("nan")), (5, 6, np.float32(-0.5)), (7, 7, np.float32(1.0)),
                    (8, 9, np.float32("-inf"))):
        W = base.copy()
        W[r, c] = v
        with pytest.raises(btas.BtasError) as ei:
            btas.apsp_paths(dev(W))
        assert ei.value.status == 1
    torch.cuda.synchronize()


@pytest.mark.parametrize("dtype", ["i32", "f32"])
@pytest.mark.parametrize("n", [8, 9, 31, 65, 130, 300, 513])
def test_argmin_matches_oracle(btas, oracle_mod, n, dtype):
    """The argmin squaring at sizes that leave ragged row, column and k edges
    and a group of 8 k cut by n: distances bit for bit and next hops equal to
    the oracle's.  int32 weights 1..20 (many ties, keyed squaring off; the
    int32 kernel mixes two add forms across columns) and binary32 weights
    U[0, 1) (rounding in play)."""
    if dtype == "i32":
        W = gen.random_graph(500 + n, n, n, 0.08 if n > 10 else 0.4, 1, 20)
    else:
        W = _f32_graph(600 + n, n, 0.08 if n > 10 else 0.4, False)
    d_ref, n_ref = oracle_mod.apsp_paths(W)
    with env(BTAS_PATHS_NO_KEYED="1"):
        D, Nx = btas.apsp_paths(dev(W))
    np.testing.assert_array_equal(bits(host(D)), bits(d_ref))
    np.testing.assert_array_equal(host(Nx), n_ref)


@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_argmin_large(btas, oracle_mod, dtype):
    """n = 2100 (32 full tiles and a ragged one per side) on the argmin
    kernel.  Sampled distance rows equal the oracle's Dijkstra rows (integer
    weights, exact in binary32 too) and sampled next-hop walks are shortest
    paths.  For int32 the next-hop matrix also equals the keyed squaring's,
    which gets the smallest minimising k from a plain product of encoded
    keys instead of from group records."""
    n = 2100
    Wi = gen.random_graph(700, n, n, 0.01, 1, 9)
    W = Wi if dtype == "i32" else np.where(Wi == INF, np.float32(np.inf), Wi.astype(np.float32)).astype(np.float32)
    with env(BTAS_PATHS_NO_KEYED="1"):
        D, Nx = btas.apsp_paths(dev(W))
    D, Nx = host(D), host(Nx)
    if dtype == "i32":
        with env(BTAS_PATHS_NO_KEYED="0"):
            Dk, Nk = btas.apsp_paths(dev(W))
        np.testing.assert_array_equal(D, host(Dk))
        np.testing.assert_array_equal(Nx, host(Nk))
    srcs = [0, 1, 777, 1500, n - 1]
    rows = oracle_mod.dijkstra_rows(Wi, srcs)
    Dr = D[srcs]
    if dtype == "f32":
        Dr = np.where(np.isinf(Dr), INF, Dr).astype(np.int32)
    np.testing.assert_array_equal(Dr, rows)
    rng = np.random.default_rng(1)
    for _ in range(300):
        i, j = (int(x) for x in rng.integers(0, n, 2))
        if (np.isinf(D[i, j]) if dtype == "f32" else D[i, j] == INF):
            assert Nx[i, j] == -1
            continue
        v, tot, steps = i, 0, 0
        while v != j:
            u = int(Nx[v, j])
            tot += int(Wi[v, u])
            v = u
            steps += 1
            assert steps <= n
        assert tot == int(D[i, j])


@pytest.mark.parametrize("dtype", ["i32", "f32"])
def test_above_the_key_range_n8200(btas, oracle_mod, dtype):
    """n = 8200, above the keyed squaring's n <= 8192: every squaring runs on
    the argmin kernel by default.  Sampled distance rows equal the oracle's
    Dijkstra rows and sampled next-hop walks are shortest paths."""
    n = 8200
    Wi = gen.random_graph(710, n, n, 0.002, 1, 9)
    W = Wi if dtype == "i32" else np.where(Wi == INF, np.float32(np.inf), Wi.astype(np.float32)).astype(np.float32)
    D, Nx = btas.apsp_paths(dev(W))
    D, Nx = host(D), host(Nx)
    srcs = [0, 4099, n - 1]
    rows = oracle_mod.dijkstra_rows(Wi, srcs)
    Dr = D[srcs]
    if dtype == "f32":
        Dr = np.where(np.isinf(Dr), INF, Dr).astype(np.int32)
    np.testing.assert_array_equal(Dr, rows)
    rng = np.random.default_rng(2)
    for _ in range(200):
        i, j = (int(x) for x in rng.integers(0, n, 2))
        if (np.isinf(D[i, j]) if dtype == "f32" else D[i, j] == INF):
            assert Nx[i, j] == -1
            continue
        v, tot, steps = i, 0, 0
        while v != j:
            u = int(Nx[v, j])
            tot += int(Wi[v, u])
            v = u
            steps += 1
            assert steps <= n
        assert tot == int(D[i, j])
