"""Blocked Floyd-Warshall on the GPU equals Algorithm 2 (oracle) and the
squaring APSP, including ragged sizes around the 128-wide tiles."""
import numpy as np
import pytest

import gen
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


@pytest.mark.parametrize("n", [1, 2, 5, 127, 128, 129, 255, 300, 513])
def test_blocked_fw_equals_oracle(btas, oracle_mod, n):
    W = gen.random_graph(31, n, n, 0.05 if n > 10 else 0.5, 0, 100)
    ref = oracle_mod.floyd_warshall(W)
    np.testing.assert_array_equal(host(btas.apsp_fw(dev(W))), ref)
    t = dev(W)
    btas.apsp_fw(t, out=t)
    np.testing.assert_array_equal(host(t), ref)


def test_blocked_fw_equals_squaring_large(btas, oracle_mod):
    n = 2048
    W = gen.random_graph(gen.BASE_SEED, 77, n, 0.01, 1, 1000)
    Wd = dev(W)
    D1 = host(btas.apsp_fw(Wd))
    D2 = host(btas.apsp(Wd))
    np.testing.assert_array_equal(D1, D2)
    srcs = gen.sample_indices(gen.BASE_SEED, 78, 16, n)
    np.testing.assert_array_equal(D1[srcs], oracle_mod.dijkstra_rows(W, srcs))
