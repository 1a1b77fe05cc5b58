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


class env:
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


@pytest.mark.parametrize("ahead", ["0", "1"])
@pytest.mark.parametrize("packed", ["0", "1"])
@pytest.mark.parametrize("whi", [100, 10 ** 6])
@pytest.mark.parametrize("n", [1, 2, 5, 127, 128, 129, 255, 300, 513])
def test_blocked_fw_equals_oracle(btas, oracle_mod, n, whi, packed, ahead):
    """Small weights: phase 3 runs packed (u16x2) where the panels allow it;
    weights up to 10^6: it stays on the int32 kernel; BTAS_FW_NO_U16=1
    forces int32 throughout.  With three or more pivot blocks, phases 1-2 of
    the next block run ahead on a second stream (BTAS_FW_NO_LOOKAHEAD=1: one
    stream, phases in order).  Same bits every time."""
    W = gen.random_graph(31, n, n, 0.05 if n > 10 else 0.5, 0, whi)
    ref = oracle_mod.floyd_warshall(W)
    with env(BTAS_FW_NO_U16="0" if packed == "1" else "1", BTAS_FW_NO_LOOKAHEAD="0" if ahead == "1" else "1"):
        np.testing.assert_array_equal(host(btas.apsp_fw(dev(W))), ref)
        t = dev(W)
        btas.apsp_fw(t, out=t)
    np.testing.assert_array_equal(host(t), ref)


def test_fw_switches_to_packed_mid_solve(btas, oracle_mod):
    """Large weights on the edges into early vertices only: the first pivot
    blocks' panels exceed the packed bound, later ones do not -- both phase-3
    kernels run within one solve, with the oracle's result."""
    n = 520
    W = gen.random_graph(32, n, n, 0.03, 1, 50)
    big = np.where((W[:, :130] != gen.INF_I32) & (np.arange(n)[:, None] != np.arange(130)[None, :]),
                   W[:, :130] + 20000, W[:, :130])
    W[:, :130] = big
    ref = oracle_mod.floyd_warshall(W)
    np.testing.assert_array_equal(host(btas.apsp_fw(dev(W))), ref)


def test_blocked_fw_equals_squaring_large(btas, oracle_mod):
    n = 2048
    W = gen.random_graph(gen.BASE_SEED, 77, n, 0.01, 1, 1000)
    Wd = dev(W)
    D1 = host(btas.apsp_fw(Wd))
    D2 = host(btas.apsp(Wd))
    np.testing.assert_array_equal(D1, D2)
    srcs = gen.sample_indices(gen.BASE_SEED, 78, 16, n)
    np.testing.assert_array_equal(D1[srcs], oracle_mod.dijkstra_rows(W, srcs))
