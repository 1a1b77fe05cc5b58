"""Pins for the oracle's tropical matrix product (Eq. 1-4; the matrix-product
listing of Sec. IV).  Each check comes from outside the oracle: hand-worked
fixtures, closed forms, semiring laws, IEEE rounding facts."""
import numpy as np
import pytest

import gen
from golden import as_f32, as_i32, load

INF = 0x3FFFFFFF
NINF = -0x3FFFFFFF
MIN, MAX = 0, 1


@pytest.mark.parametrize("name,sr", [
    ("tgemm_i32_minplus_2x3x2.txt", MIN),
    ("tgemm_i32_maxplus_2x3x2.txt", MAX),
    ("tgemm_i32_minplus_negative_2x2x2.txt", MIN),
])
def test_hand_worked_int(oracle_mod, name, sr):
    g = load(name)
    C = oracle_mod.tgemm(sr, as_i32(g["A"]), as_i32(g["B"]))
    np.testing.assert_array_equal(C, as_i32(g["C"]))


def test_hand_worked_f32(oracle_mod):
    g = load("tgemm_f32_minplus_2x2x2.txt")
    C = oracle_mod.tgemm(MIN, as_f32(g["A"]), as_f32(g["B"]))
    np.testing.assert_array_equal(C, as_f32(g["C"]))


def test_round_to_nearest_even(oracle_mod):
    g = load("tgemm_f32_rounding_1x2x1.txt")
    A, B = as_f32(g["A"]), as_f32(g["B"])
    assert oracle_mod.tgemm(MIN, A, B).view(np.uint32)[0, 0] == as_f32(g["Cmin"]).view(np.uint32)[0, 0]
    assert oracle_mod.tgemm(MAX, A, B).view(np.uint32)[0, 0] == as_f32(g["Cmax"]).view(np.uint32)[0, 0]
    assert as_f32(g["Cmax"])[0, 0] == np.float32(1.0) + np.float32(2.0 ** -22)


def _rand_i32(seed, shape, lo=-1000, hi=1000, p_inf=0.0, inf=INF):
    v = gen.uniform_int(seed, 1, shape, lo, hi)
    if p_inf:
        u = gen.uniform_unit_f64(seed, 2, np.arange(v.size, dtype=np.uint64)).reshape(shape)
        v = np.where(u < p_inf, inf, v).astype(np.int32)
    return v


def test_k1_is_outer_sum(oracle_mod):
    """With k = 1 the product is the outer (.)-product a_i + b_j (closed form)."""
    a = _rand_i32(3, (7, 1))
    b = _rand_i32(4, (1, 5))
    for sr in (MIN, MAX):
        C = oracle_mod.tgemm(sr, a, b)
        np.testing.assert_array_equal(C, a.astype(np.int64) + b.astype(np.int64))


def test_k0_gives_identity_and_accumulate_keeps(oracle_mod):
    A = np.zeros((3, 0), np.int32)
    B = np.zeros((0, 4), np.int32)
    assert (oracle_mod.tgemm(MIN, A, B) == INF).all()
    assert (oracle_mod.tgemm(MAX, A, B) == NINF).all()
    C0 = _rand_i32(5, (3, 4))
    np.testing.assert_array_equal(oracle_mod.tgemm(MIN, A, B, C0), C0)


def _identity(n, sr):
    E = np.full((n, n), INF if sr == MIN else NINF, np.int32)
    np.fill_diagonal(E, 0)
    return E


@pytest.mark.parametrize("sr", [MIN, MAX])
def test_identity_is_neutral_and_zero_absorbs(oracle_mod, sr):
    inf = INF if sr == MIN else NINF
    A = _rand_i32(6, (9, 13), p_inf=0.2, inf=inf)
    np.testing.assert_array_equal(oracle_mod.tgemm(sr, _identity(9, sr), A), A)
    np.testing.assert_array_equal(oracle_mod.tgemm(sr, A, _identity(13, sr)), A)
    Z = np.full((13, 4), inf, np.int32)
    assert (oracle_mod.tgemm(sr, A, Z) == inf).all()


@pytest.mark.parametrize("sr", [MIN, MAX])
def test_associativity_int(oracle_mod, sr):
    inf = INF if sr == MIN else NINF
    A = _rand_i32(7, (6, 8), -100, 100, 0.2, inf)
    B = _rand_i32(8, (8, 5), -100, 100, 0.2, inf)
    C = _rand_i32(9, (5, 7), -100, 100, 0.2, inf)
    left = oracle_mod.tgemm(sr, oracle_mod.tgemm(sr, A, B), C)
    right = oracle_mod.tgemm(sr, A, oracle_mod.tgemm(sr, B, C))
    np.testing.assert_array_equal(left, right)


def test_minplus_maxplus_duality(oracle_mod):
    """max-plus(A, B) = -min-plus(-A, -B), with INF <-> -INF (exact)."""
    A = _rand_i32(10, (11, 17), p_inf=0.3, inf=NINF)
    B = _rand_i32(11, (17, 6), p_inf=0.3, inf=NINF)
    mx = oracle_mod.tgemm(MAX, A, B)
    mn = oracle_mod.tgemm(MIN, -A, -B)
    np.testing.assert_array_equal(mx, -mn)
    Af = gen.uniform_f32(12, 1, (11, 17))
    Bf = gen.uniform_f32(13, 1, (17, 6))
    np.testing.assert_array_equal(oracle_mod.tgemm(MAX, Af, Bf), -oracle_mod.tgemm(MIN, -Af, -Bf))


@pytest.mark.parametrize("sr", [MIN, MAX])
def test_translation_invariance_int(oracle_mod, sr):
    """(A + a) (x) (B + b) = (A (x) B) + a + b on finite entries, identity
    entries staying the identity (each term shifts by a + b, and min/max
    commute with a common shift); the law the packed int32 path relies on."""
    inf = INF if sr == MIN else NINF
    A = _rand_i32(14, (9, 13), -500, 500, 0.25, inf)
    B = _rand_i32(15, (13, 7), -500, 500, 0.25, inf)
    A[2, :] = inf  # a row with no finite term: its outputs stay the identity
    a, b = -377, 1234
    As = np.where(A == inf, inf, A + a).astype(np.int32)
    Bs = np.where(B == inf, inf, B + b).astype(np.int32)
    C = oracle_mod.tgemm(sr, A, B)
    Cs = oracle_mod.tgemm(sr, As, Bs)
    np.testing.assert_array_equal(Cs, np.where(C == inf, inf, C + a + b))
    assert (C == inf).any() and (C != inf).any()


@pytest.mark.parametrize("dt", ["i32", "f32"])
@pytest.mark.parametrize("sr", [MIN, MAX])
def test_split_k_partials_combine(oracle_mod, dt, sr):
    """(+) is associative, commutative and idempotent, so the (+) of partial
    products over a split of k equals the whole product, for ints and FP32."""
    if dt == "i32":
        inf = INF if sr == MIN else NINF
        A = _rand_i32(14, (5, 23), p_inf=0.2, inf=inf)
        B = _rand_i32(15, (23, 9), p_inf=0.2, inf=inf)
    else:
        A = gen.uniform_f32(14, 1, (5, 23))
        B = gen.uniform_f32(15, 1, (23, 9))
    whole = oracle_mod.tgemm(sr, A, B)
    p1 = oracle_mod.tgemm(sr, A[:, :10], B[:10])
    both = oracle_mod.tgemm(sr, A[:, 10:], B[10:], p1)
    np.testing.assert_array_equal(whole, both)


@pytest.mark.parametrize("sr", [MIN, MAX])
def test_f32_equals_rounded_exact(oracle_mod, sr):
    """Rounding is monotone, so min_k fl(a+b) = fl(min_k (a+b)): the FP32
    product equals the fp64-exact product (two binary32 values sum exactly
    in binary64) rounded once to binary32."""
    A = gen.uniform_f32(16, 1, (12, 40)) * np.float32(3.0) - np.float32(1.0)
    B = gen.uniform_f32(17, 1, (40, 10)) * np.float32(1e-3)
    C = oracle_mod.tgemm(sr, A, B)
    s = A.astype(np.float64)[:, :, None] + B.astype(np.float64)[None, :, :]
    exact = s.min(axis=1) if sr == MIN else s.max(axis=1)
    np.testing.assert_array_equal(C.view(np.uint32), exact.astype(np.float32).view(np.uint32))


def test_nonsquare_operands_not_transposed(oracle_mod):
    """A row-major 3x5 times 5x2 with distinct entries: every C[i][j] is the
    minimum over exactly the pairs (A[i][l], B[l][j])."""
    A = np.arange(15, dtype=np.int32).reshape(3, 5) * 7 % 11
    B = np.arange(10, dtype=np.int32).reshape(5, 2) * 5 % 13
    C = oracle_mod.tgemm(MIN, A, B)
    for i in range(3):
        for j in range(2):
            assert C[i, j] == min(int(A[i, l]) + int(B[l, j]) for l in range(5))


def test_u16_saturates_and_matches_int32(oracle_mod):
    """16-bit product = min(INF16, int32 product) when INF16 maps to a large
    int32 sentinel; finite sums below INF16 are exact."""
    A = gen.uniform_int(18, 1, (20, 30), 0, 0x7FFF).astype(np.uint16)
    B = gen.uniform_int(19, 1, (30, 25), 0, 0x7FFF).astype(np.uint16)
    C16 = oracle_mod.tgemm_u16(A, B).astype(np.int64)
    a32 = np.where(A == 0x7FFF, INF, A.astype(np.int64)).astype(np.int32)
    b32 = np.where(B == 0x7FFF, INF, B.astype(np.int64)).astype(np.int32)
    C32 = oracle_mod.tgemm(MIN, a32, b32).astype(np.int64)
    np.testing.assert_array_equal(C16, np.minimum(C32, 0x7FFF))
    # hand case: 0x4000 + 0x4000 saturates, 3 + 4 does not
    a = np.array([[0x4000, 3]], np.uint16)
    b = np.array([[0x4000], [4]], np.uint16)
    assert oracle_mod.tgemm_u16(a, b)[0, 0] == 7
    assert oracle_mod.tgemm_u16(a[:, :1], b[:1])[0, 0] == 0x7FFF


def test_threads_do_not_change_results(oracle_mod):
    A = _rand_i32(20, (33, 40), p_inf=0.1)
    B = _rand_i32(21, (40, 17), p_inf=0.1)
    oracle_mod.set_threads(1)
    c1 = oracle_mod.tgemm(MIN, A, B)
    oracle_mod.set_threads(4)
    c4 = oracle_mod.tgemm(MIN, A, B)
    oracle_mod.set_threads(1)
    np.testing.assert_array_equal(c1, c4)
