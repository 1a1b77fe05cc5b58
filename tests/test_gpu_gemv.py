"""Level 2 (tropical gemv) and Bellman-Ford SSSP by repeated vector-matrix
products, against the oracle (bit-exact) and Dijkstra."""
import numpy as np
import pytest

import gen
from gpu_util import INF, bits, dev, f32_matrix, host, int_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_gemv_shapes(btas, oracle_mod, dt, sr, trans):
    mk = int_matrix if dt == "i32" else f32_matrix
    for (m, n) in [(1, 1), (3, 5), (33, 130), (257, 63), (1000, 1001), (64, 4096)]:
        A = mk(300 + m, (m, n), sr)
        x = mk(400 + n, ((m if trans else n),), sr)
        ref = oracle_mod.gemv(sr, A, x, trans=trans)
        y = host(btas.gemv(dev(A), dev(x), sr, trans=trans))
        np.testing.assert_array_equal(bits(y), bits(ref), err_msg=f"{dt} sr={sr} trans={trans} {m}x{n}")
        y0 = mk(500 + m, ((n if trans else m),), sr)
        yd = dev(y0)
        btas.gemv(dev(A), dev(x), sr, trans=trans, out=yd, accumulate=True)
        np.testing.assert_array_equal(bits(host(yd)), bits(oracle_mod.gemv(sr, A, x, trans=trans, y=y0)))


def test_gemv_strided_and_unaligned(btas, oracle_mod):
    import torch
    A = int_matrix(7, (70, 91), 0)
    Abig = dev(np.pad(A, ((0, 0), (0, 3))))
    x = int_matrix(8, (91,), 0)
    ref = oracle_mod.gemv(0, A, x)
    np.testing.assert_array_equal(host(btas.gemv(Abig[:, :91], dev(x), 0)), ref)


@pytest.fixture(params=["coop", "grouped"])
def sssp_mode(request):
    """coop: all relaxations in one cooperative launch (the default);
    grouped: BTAS_SSSP_NO_COOP=1, one launch per relaxation in gated groups."""
    import os
    old = os.environ.get("BTAS_SSSP_NO_COOP")
    os.environ["BTAS_SSSP_NO_COOP"] = "1" if request.param == "grouped" else "0"
    yield request.param
    if old is None:
        del os.environ["BTAS_SSSP_NO_COOP"]
    else:
        os.environ["BTAS_SSSP_NO_COOP"] = old


@pytest.mark.parametrize("n", [1, 2, 50, 777, 1027, 4096])
def test_sssp_matches_dijkstra_and_oracle(btas, oracle_mod, n, sssp_mode):
    W = gen.random_graph(gen.BASE_SEED, 90 + n % 7, n, 0.01 if n > 1000 else 0.1, 1, 1000)
    Wd = dev(W)
    for src in sorted({0, n // 3, n - 1}):
        d, info = btas.sssp(Wd, src, info=True)
        d = host(d)
        np.testing.assert_array_equal(d, oracle_mod.dijkstra_rows(W, [src])[0])
        if n <= 777:
            ref, steps = oracle_mod.sssp(W, src)
            np.testing.assert_array_equal(d, ref)
            assert info["iterations"] == steps


@pytest.mark.parametrize("n", [2, 9, 17, 20, 33])
def test_sssp_long_chains(btas, oracle_mod, n, sssp_mode):
    """A directed path needs n - 1 changing relaxations: as many grid
    barriers in the cooperative kernel; several groups of relaxations
    enqueued between read-backs, the last one partial, in the grouped mode."""
    W = np.full((n, n), INF, np.int32)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 3
    W[n - 1, 0] = 5  # a back edge closes a cycle and changes nothing from source 0
    d, info = btas.sssp(dev(W), 0, info=True)
    ref, steps = oracle_mod.sssp(W, 0)
    np.testing.assert_array_equal(host(d), ref)
    assert info["iterations"] == steps
    d, info = btas.sssp(dev(W), n - 1, info=True)
    ref, steps = oracle_mod.sssp(W, n - 1)
    np.testing.assert_array_equal(host(d), ref)
    assert info["iterations"] == steps


@pytest.mark.parametrize("where", ["weight", "diagonal"])
def test_sssp_domain_violation(btas, sssp_mode, where):
    """A negative weight or a non-zero diagonal entry is reported
    (BTAS_ERR_ARG) and dist is left as it was; the cooperative kernel finds it
    during its first product."""
    import torch
    n = 300
    W = gen.random_graph(gen.BASE_SEED, 97, n, 0.05, 1, 100)
    if where == "weight":
        W[17, 250] = -4
    else:
        W[123, 123] = 9
    Wd = dev(W)
    dist = torch.full((n,), 55, dtype=torch.int32, device="cuda")
    it = __import__("ctypes").c_int(0)
    st = torch.cuda.current_stream().cuda_stream
    rc = btas.lib().btas_sssp(n, Wd.data_ptr(), 0, dist.data_ptr(), __import__("ctypes").addressof(it), st)
    torch.cuda.synchronize()
    assert rc == 1 and "outside the domain" in btas.last_error()
    assert (host(dist) == 55).all()
