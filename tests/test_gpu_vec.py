"""GPU parity of the tropical vector operations against the oracle."""
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


@pytest.mark.parametrize("n", [0, 1, 5, 1000, 100003, 3_000_001])
@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_dot(btas, oracle_mod, dt, sr, n):
    mk = int_matrix if dt == "i32" else f32_matrix
    x = mk(40 + n % 97, (max(n, 1) * 2,), sr)
    y = mk(41 + n % 89, (max(n, 1),), sr)
    ref = oracle_mod.dot(sr, x, y, incx=2, incy=1, n=n)
    r = host(btas.dot(dev(x), dev(y), sr, incx=2, incy=1, n=n))
    assert bits(np.array([r]))[0] == bits(np.array([ref]))[0]


@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_axpy_add_mul(btas, oracle_mod, dt, sr):
    mk = int_matrix if dt == "i32" else f32_matrix
    n = 123457
    x = mk(50, (2 * n,), sr)
    y = mk(51, (n,), sr)
    alpha = 17 if dt == "i32" else 0.375
    ref = oracle_mod.axpy(sr, alpha, x, y, incx=2, incy=1, n=n)
    yd = dev(y)
    btas.axpy(alpha, dev(x), yd, sr, incx=2, incy=1, n=n)
    np.testing.assert_array_equal(bits(host(yd)), bits(ref))
    x1 = np.ascontiguousarray(x[:n])
    np.testing.assert_array_equal(bits(host(btas.add(dev(x1), dev(y), sr))), bits(oracle_mod.add(sr, x1, y)))
    np.testing.assert_array_equal(bits(host(btas.mul(dev(x1), dev(y), sr))), bits(oracle_mod.mul(sr, x1, y)))
