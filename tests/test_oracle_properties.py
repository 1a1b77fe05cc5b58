"""Property-based pins of the oracle (hypothesis; skipped where it is not
installed).  Each property is a law of the semirings (Eq. 1-4) or of
shortest paths that a plausible mistake in the oracle would break: a dropped
INF check, a wrong comparison direction, a transposed operand, an off-by-one
in the squaring count."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

INF = 0x3FFFFFFF
NINF = -0x3FFFFFFF
SETTINGS = settings(max_examples=60, deadline=None)


def _int_matrix(draw, rows, cols, sr, lo=-50, hi=50):
    ident = INF if sr == 0 else NINF
    vals = draw(st.lists(st.one_of(st.integers(lo, hi), st.just(ident)), min_size=rows * cols,
                         max_size=rows * cols))
    return np.array(vals, dtype=np.int32).reshape(rows, cols)


@st.composite
def product_triple(draw):
    sr = draw(st.integers(0, 1))
    m, k, n = draw(st.integers(1, 6)), draw(st.integers(1, 6)), draw(st.integers(1, 6))
    A = _int_matrix(draw, m, k, sr)
    B = _int_matrix(draw, k, n, sr)
    C = _int_matrix(draw, k, n, sr)
    return sr, A, B, C


def _oplus(sr, X, Y):
    return np.minimum(X, Y) if sr == 0 else np.maximum(X, Y)


@SETTINGS
@given(product_triple())
def test_distributivity(oracle_mod, t):
    """A (x) (B (+) C) = (A (x) B) (+) (A (x) C)."""
    sr, A, B, C = t
    left = oracle_mod.tgemm(sr, A, _oplus(sr, B, C))
    right = _oplus(sr, oracle_mod.tgemm(sr, A, B), oracle_mod.tgemm(sr, A, C))
    np.testing.assert_array_equal(left, right)


@SETTINGS
@given(product_triple())
def test_monotone_in_each_operand(oracle_mod, t):
    """Improving an operand entry (smaller for min-plus, larger for max-plus)
    can only improve the product, entry by entry."""
    sr, A, B, _ = t
    better = np.where(B == (INF if sr == 0 else NINF), B, B - 3 if sr == 0 else B + 3).astype(np.int32)
    P, Q = oracle_mod.tgemm(sr, A, B), oracle_mod.tgemm(sr, A, better)
    assert (Q <= P).all() if sr == 0 else (Q >= P).all()


@SETTINGS
@given(product_triple())
def test_transpose_rule(oracle_mod, t):
    """(A (x) B)^T = B^T (x) A^T (the semiring is commutative)."""
    sr, A, B, _ = t
    np.testing.assert_array_equal(oracle_mod.tgemm(sr, A, B).T,
                                  oracle_mod.tgemm(sr, np.ascontiguousarray(B.T), np.ascontiguousarray(A.T)))


@st.composite
def graph(draw):
    n = draw(st.integers(1, 7))
    W = np.full((n, n), INF, np.int32)
    for i in range(n):
        for j in range(n):
            if i != j and draw(st.booleans()):
                W[i, j] = draw(st.integers(0, 20))
    np.fill_diagonal(W, 0)
    return W


@SETTINGS
@given(graph())
def test_apsp_methods_and_invariants(oracle_mod, W):
    """Squaring = Floyd-Warshall = brute force over simple paths = Dijkstra;
    the result is a fixpoint of the squaring, has a zero diagonal, never
    exceeds W, and satisfies the triangle inequality."""
    n = W.shape[0]
    D = oracle_mod.apsp_squaring(W)
    np.testing.assert_array_equal(D, oracle_mod.floyd_warshall(W))
    np.testing.assert_array_equal(D, oracle_mod.bruteforce_apsp(W))
    np.testing.assert_array_equal(D, oracle_mod.dijkstra_rows(W, np.arange(n)))
    np.testing.assert_array_equal(oracle_mod.tgemm(0, D, D), D)
    assert (np.diag(D) == 0).all() and (D <= W).all()
    fin = D < INF
    for k in range(n):
        via = np.where(fin[:, [k]] & fin[[k], :], D[:, [k]].astype(np.int64) + D[[k], :], INF)
        assert (D <= via).all()
