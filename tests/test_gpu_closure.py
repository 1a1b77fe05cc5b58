"""Tropical closure A* = E (+) A (+) A^2 (+) ... by repeated squaring:
min-plus with negative edges (no negative cycle) vs Floyd-Warshall on
E (+) A; max-plus by duality; FP32 APSP vs the oracle's fp32 squaring
sequence; divergence (negative / positive cycle) is reported."""
import numpy as np
import pytest

import gen
from gpu_util import INF, NINF, bits, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def _potential_graph(seed, n, p):
    """Weights w(i,j) + pi(i) - pi(j) with w >= 0: negative edges, but every
    cycle keeps its non-negative weight."""
    W = gen.random_graph(seed, 1, n, p, 0, 50).astype(np.int64)
    pi = gen.uniform_int(seed, 9, (n,), 0, 40).astype(np.int64)
    A = np.where(W == INF, INF, W + pi[:, None] - pi[None, :])
    np.fill_diagonal(A, gen.uniform_int(seed, 10, (n,), 0, 5))  # arbitrary non-negative diagonal
    return A.astype(np.int32)


def _eplus(A, sr):
    B = A.copy()
    d = np.diag(B)
    np.fill_diagonal(B, np.minimum(d, 0) if sr == 0 else np.maximum(d, 0))
    return B


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 130, 300])
def test_minplus_negative_edges_vs_floyd_warshall(btas, oracle_mod, n):
    A = _potential_graph(100 + n, n, 0.2 if n > 3 else 0.7)
    ref = oracle_mod.floyd_warshall(_eplus(A, 0))
    out = host(btas.closure(dev(A), "min"))
    np.testing.assert_array_equal(out, ref)
    # max-plus by duality: maxplus*(-A) = -(minplus*(A)), INF <-> -INF
    Am = np.where(A == INF, NINF, -A.astype(np.int64)).astype(np.int32)
    outm = host(btas.closure(dev(Am), "max"))
    np.testing.assert_array_equal(outm, np.where(ref == INF, NINF, -ref.astype(np.int64)).astype(np.int32))


@pytest.mark.parametrize("n", [5, 64, 257])
def test_fp32_apsp_equals_oracle_squaring(btas, oracle_mod, n):
    W = gen.random_graph(7, n, n, 0.1, 1, 100)
    Wf = np.where(W == INF, np.inf, gen.uniform_f32(8, n, (n, n)) * np.float32(3.0) + np.float32(0.001))
    np.fill_diagonal(Wf, 0.0)
    Wf = Wf.astype(np.float32)
    D = Wf.copy()
    for _ in range(oracle_mod.apsp_squarings(n)):
        D = oracle_mod.tgemm(0, D, D)
    out = host(btas.closure(dev(Wf), "min"))
    np.testing.assert_array_equal(bits(out), bits(D))


def test_cycle_is_reported(btas):
    import paper_1701_04733_gb300 as b_mod
    A = _potential_graph(5, 40, 0.2)
    A[3, 7] = -1000  # a negative cycle through 3 -> 7 -> ... -> 3 once 7 reaches 3
    A[7, 3] = 0
    with pytest.raises(b_mod.BtasError):
        btas.closure(dev(A), "min")
    Af = np.array([[0.0, 1.0], [1.0, 0.0]], np.float32)
    with pytest.raises(b_mod.BtasError):
        btas.closure(dev(Af), "max")  # positive cycle 0 -> 1 -> 0 of weight 2
