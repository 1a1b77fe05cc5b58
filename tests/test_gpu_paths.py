"""APSP with path reconstruction: distances and the next-hop matrix are
bit-identical to the oracle's squaring with the smallest-minimising-k rule,
and every next-hop walk is a shortest path."""
import numpy as np
import pytest

import gen
from golden import as_i32, load
from gpu_util import INF, dev, host

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


@pytest.mark.parametrize("n", [1, 2, 3, 31, 64, 65, 200, 513])
def test_matches_oracle_and_walks_are_shortest(btas, oracle_mod, n):
    W = gen.random_graph(21, n, n, 0.08 if n > 10 else 0.5, 1, 20)
    ref_d, ref_n = oracle_mod.apsp_paths(W)
    for early in (True, False):
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
