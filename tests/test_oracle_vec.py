"""Pins for the oracle's tropical vector operations (the "standard vector
operations" of the abstract and Sec. III, built from Eq. 1-4)."""
import numpy as np
import pytest

import gen

INF = 0x3FFFFFFF
NINF = -0x3FFFFFFF


def test_dot_hand_worked(oracle_mod):
    x = np.array([3, INF, -2, 7], np.int32)
    y = np.array([1, 0, 5, INF], np.int32)
    # min(3+1, INF, -2+5, INF) = 3
    assert oracle_mod.dot(0, x, y) == 3
    xm = np.array([3, NINF, -2, 7], np.int32)
    ym = np.array([1, 0, 5, NINF], np.int32)
    # max(4, -INF, 3, -INF) = 4
    assert oracle_mod.dot(1, xm, ym) == 4
    assert oracle_mod.dot(0, x[:0], y[:0]) == INF
    assert oracle_mod.dot(1, x[:0], y[:0]) == NINF


def test_dot_strided_hand_worked(oracle_mod):
    x = np.array([1, 100, 2, 100, 3], np.int32)   # stride 2 -> 1, 2, 3
    y = np.array([9, 8, 7], np.int32)             # stride 1
    assert oracle_mod.dot(0, x, y, incx=2, incy=1, n=3) == min(1 + 9, 2 + 8, 3 + 7)
    assert oracle_mod.dot(1, x, y, incx=2, incy=1, n=3) == 10


def test_dot_is_1xn_times_nx1_product(oracle_mod):
    """dot(x, y) is the 1 x n by n x 1 tropical matrix product."""
    x = gen.uniform_f32(1, 1, (257,))
    y = gen.uniform_f32(2, 1, (257,))
    for sr in (0, 1):
        assert oracle_mod.dot(sr, x, y) == oracle_mod.tgemm(sr, x[None, :], y[:, None])[0, 0]


def test_axpy_hand_worked(oracle_mod):
    x = np.array([1, 5, INF], np.int32)
    y = np.array([4, 2, 6], np.int32)
    # y_i <- min(y_i, 2 + x_i) = [3, 2, 6]
    np.testing.assert_array_equal(oracle_mod.axpy(0, 2, x, y), [3, 2, 6])
    np.testing.assert_array_equal(oracle_mod.axpy(1, 2, x[:2], y[:2]), [4, 7])


def test_axpy_unit_alpha_is_add(oracle_mod):
    """alpha = 0 is the (.)-identity, so axpy reduces to y (+) x."""
    x = gen.uniform_int(3, 1, (100,), -50, 50)
    y = gen.uniform_int(4, 1, (100,), -50, 50)
    for sr in (0, 1):
        np.testing.assert_array_equal(oracle_mod.axpy(sr, 0, x, y), oracle_mod.add(sr, x, y))


def test_add_mul_hand_worked(oracle_mod):
    x = np.array([1, INF, -3], np.int32)
    y = np.array([2, 5, INF], np.int32)
    np.testing.assert_array_equal(oracle_mod.add(0, x, y), [1, 5, -3])
    np.testing.assert_array_equal(oracle_mod.mul(0, x, y), [3, INF, INF])
    xf = np.array([0.5, np.inf], np.float32)
    yf = np.array([0.25, 1.0], np.float32)
    np.testing.assert_array_equal(oracle_mod.add(0, xf, yf), [0.25, 1.0])
    np.testing.assert_array_equal(oracle_mod.add(1, xf, yf), [0.5, np.inf])
    np.testing.assert_array_equal(oracle_mod.mul(0, xf, yf), [0.75, np.inf])


def test_add_is_commutative_idempotent(oracle_mod):
    x = gen.uniform_f32(5, 1, (64,))
    y = gen.uniform_f32(6, 1, (64,))
    for sr in (0, 1):
        np.testing.assert_array_equal(oracle_mod.add(sr, x, y), oracle_mod.add(sr, y, x))
        np.testing.assert_array_equal(oracle_mod.add(sr, x, x), x)


def test_gemv_hand_worked(oracle_mod):
    A = np.array([[1, 5, INF], [0, 2, 3]], np.int32)
    x = np.array([4, 1, 0], np.int32)
    # y0 = min(1+4, 5+1, INF+0) = 5 ; y1 = min(0+4, 2+1, 3+0) = 3
    np.testing.assert_array_equal(oracle_mod.gemv(0, A, x), [5, 3])
    # trans: y_j = min_i x_i + A[i][j] with x = (2, 1)
    xt = np.array([2, 1], np.int32)
    # y0 = min(2+1, 1+0) = 1 ; y1 = min(2+5, 1+2) = 3 ; y2 = min(2+INF, 1+3) = 4
    np.testing.assert_array_equal(oracle_mod.gemv(0, A, xt, trans=True), [1, 3, 4])
    # max-plus: y0 = max(1+4, 5+1) = 6 (the INF entry is a large finite here, so use a finite matrix)
    Af = np.array([[1, 5], [0, 2]], np.int32)
    np.testing.assert_array_equal(oracle_mod.gemv(1, Af, np.array([4, 1], np.int32)), [6, 4])


def test_gemv_is_one_column_product(oracle_mod):
    A = gen.uniform_f32(7, 1, (33, 21))
    x = gen.uniform_f32(8, 1, (21,))
    for sr in (0, 1):
        np.testing.assert_array_equal(oracle_mod.gemv(sr, A, x), oracle_mod.tgemm(sr, A, x[:, None])[:, 0])
        xt = gen.uniform_f32(9, 1, (33,))
        np.testing.assert_array_equal(oracle_mod.gemv(sr, A, xt, trans=True), oracle_mod.tgemm(sr, xt[None, :], A)[0])


def test_sssp_equals_dijkstra(oracle_mod):
    for n in (1, 2, 7, 50, 200):
        W = gen.random_graph(12, n, n, 0.05 if n > 10 else 0.4, 1, 50)
        for src in {0, n // 2, n - 1}:
            d, steps = oracle_mod.sssp(W, src)
            np.testing.assert_array_equal(d, oracle_mod.dijkstra_rows(W, [src])[0])
            assert 0 <= steps <= max(0, n - 1)
