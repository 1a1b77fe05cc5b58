"""The two exact shortcuts of the cooperative APSP kernel, checked on the CPU
with plain numpy on small graphs (no oracle, no GPU):

- the first squaring from edge lists: X_1[i][j] = min(W[i][j], w_ik + w_kj
  over edges (i, k), (k, j)) equals the dense product W (x) W (Sec. III's
  first squaring);
- the closure certificate: after squaring s, X_s[i][j] <= X_s[i][k] + W[k][j]
  at every entry (i, k) that squaring s lowered and every edge (k, j) holds
  exactly when X_s (x) X_s == X_s, i.e. when squaring s + 1 would change
  nothing -- so the kernel may stop without computing it.

Both are stated for non-negative weights and a zero diagonal, the domain of
the APSP routines."""
import numpy as np
import pytest

BIG = 1 << 40  # "no edge" here


def graph(rng, n, p, whi):
    W = np.where(rng.random((n, n)) < p, rng.integers(1, whi + 1, (n, n)), BIG).astype(np.int64)
    np.fill_diagonal(W, 0)
    return W


def minplus(A, B):
    C = np.min(A[:, :, None] + B[None, :, :], axis=1)
    return np.where(C >= BIG, BIG, C)


def sparse_first(W):
    n = W.shape[0]
    X = W.copy()
    edges = [[(j, int(W[k, j])) for j in range(n) if j != k and W[k, j] < BIG] for k in range(n)]
    for i in range(n):
        for k, wik in edges[i]:
            for j, wkj in edges[k]:
                X[i, j] = min(X[i, j], wik + wkj)
    return X


def certificate(W, X, Xprev):
    """True when no lowered entry (i, k) and edge (k, j) gives X[i][k] + w_kj < X[i][j]."""
    n = W.shape[0]
    for i, k in zip(*np.nonzero(X < Xprev)):
        for j in range(n):
            if j != k and W[k, j] < BIG and X[i, k] + W[k, j] < X[i, j]:
                return False
    return True


def full_certificate(W, X):
    """X (x) W >= X entrywise (every pair, not only the lowered ones)."""
    return bool((minplus(X, W) >= X).all())


CASES = [(n, p, whi) for n in (6, 13, 24, 40) for p, whi in ((0.08, 10), (0.2, 100), (0.5, 3), (0.04, 1000))]


@pytest.mark.parametrize("n,p,whi", CASES)
def test_sparse_first_squaring_is_the_product(n, p, whi):
    rng = np.random.default_rng(1000 * n + int(100 * p) + whi)
    for _ in range(3):
        W = graph(rng, n, p, whi)
        np.testing.assert_array_equal(sparse_first(W), minplus(W, W))


@pytest.mark.parametrize("n,p,whi", CASES)
def test_certificate_decides_the_next_squaring(n, p, whi):
    rng = np.random.default_rng(7 + 1000 * n + int(100 * p) + whi)
    seen = {True: 0, False: 0}
    for _ in range(4):
        W = graph(rng, n, p, whi)
        X_prev, X = W, minplus(W, W)
        for _s in range(8):
            nxt = minplus(X, X)
            fixed = bool((nxt == X).all())
            assert certificate(W, X, X_prev) == fixed
            assert full_certificate(W, X) == fixed
            seen[fixed] += 1
            if fixed:
                break
            X_prev, X = X, nxt
    assert seen[True] > 0


def test_certificate_on_a_directed_path():
    """A directed path lowers entries in every squaring: the certificate fails
    until the squaring that reaches the whole path."""
    n = 19
    W = np.full((n, n), BIG, np.int64)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 3
    X_prev, X = W, minplus(W, W)
    outcomes = []
    for _s in range(6):
        outcomes.append(certificate(W, X, X_prev))
        nxt = minplus(X, X)
        if (nxt == X).all():
            break
        X_prev, X = X, nxt
    # hops covered after squaring s: 2^s; 18 hops need s = 5
    assert outcomes == [False, False, False, False, True]
    assert X[0, n - 1] == 3 * (n - 1)


def test_a_lowered_entry_is_needed_to_fail():
    """Planted mistake: a certificate that skips the lowered entries (checks
    only the unchanged ones) would pass too early on the path graph."""
    n = 9
    W = np.full((n, n), BIG, np.int64)
    np.fill_diagonal(W, 0)
    W[np.arange(n - 1), np.arange(1, n)] = 1
    X_prev, X = W, minplus(W, W)
    unchanged_only = all(
        not (j != k and W[k, j] < BIG and X[i, k] + W[k, j] < X[i, j])
        for i in range(n) for k in range(n) if X[i, k] == X_prev[i, k] for j in range(n))
    assert unchanged_only and not certificate(W, X, X_prev)


def minplus_clamped(A, B, T):
    """The products' arithmetic: sums >= T become "no path" (BIG)."""
    C = np.min(A[:, :, None] + B[None, :, :], axis=1)
    return np.where(C >= T, BIG, C)


def certificate_clamped(W, X, Xprev, T):
    n = W.shape[0]
    for i, k in zip(*np.nonzero(X < Xprev)):
        for j in range(n):
            s = X[i, k] + W[k, j]
            if j != k and W[k, j] < BIG and s < T and s < X[i, j]:
                return False
    return True


@pytest.mark.parametrize("T", [12, 25, 60])
def test_certificate_under_the_clamp(T):
    """With the clamp at a small threshold T, so that long paths saturate to
    "no path" as they do above INF - 2^28 in the kernels, the certificate
    still holds exactly when the next clamped squaring changes nothing."""
    rng = np.random.default_rng(100 + T)
    checked = 0
    for _ in range(30):
        n = int(rng.integers(5, 20))
        W = graph(rng, n, float(rng.choice([0.1, 0.25, 0.5])), 9)
        X_prev, X = W, minplus_clamped(W, W, T)
        for _s in range(8):
            nxt = minplus_clamped(X, X, T)
            fixed = bool((nxt == X).all())
            assert certificate_clamped(W, X, X_prev, T) == fixed
            checked += 1
            if fixed:
                break
            X_prev, X = X, nxt
    assert checked > 30
