"""GPU parity of the tropical matrix product against the CPU oracle.

Bit-exact for every dtype: each term is one exact integer add or one
round-to-nearest fp32 add, and min/max does not depend on order, so every
tiling and every inner-loop variant must reproduce the oracle's bits."""
import os

import numpy as np
import pytest

import gen
from gpu_util import INF, NINF, bits, dev, f32_matrix, host, int_matrix

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (3, 5, 2), (31, 33, 17), (64, 64, 64), (129, 127, 33), (200, 300, 129), (300, 260, 70),
          (257, 513, 100), (130, 70, 1000)]
I32_VARIANTS = [{"BTAS_I32_VARIANT": "0"}, {"BTAS_I32_VARIANT": "1", "BTAS_I32_NS": "4"}, {"BTAS_I32_VARIANT": "1", "BTAS_I32_NS": "8"},
                {"BTAS_I32_VARIANT": "1", "BTAS_I32_NS": "5"}, {"BTAS_I32_VARIANT": "1", "BTAS_I32_NS": "6"}]
F32_VARIANTS = [{"BTAS_F32_VARIANT": "2"}, {"BTAS_F32_VARIANT": "3"}, {"BTAS_F32_VARIANT": "4"}]


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
        self.old = {k: os.environ.get(k) for k in self.kv}
        os.environ.update(self.kv)

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _inputs(dt, sr, m, n, k, seed):
    if dt == "i32":
        return int_matrix(seed, (m, k), sr), int_matrix(seed + 1, (k, n), sr)
    return f32_matrix(seed, (m, k), sr), f32_matrix(seed + 1, (k, n), sr)


@pytest.mark.parametrize("cfg", ["0", "2", "4"])
@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_shapes_all_variants(btas, oracle_mod, dt, sr, cfg):
    variants = I32_VARIANTS if dt == "i32" else F32_VARIANTS
    for si, (m, n, k) in enumerate(SHAPES):
        A, B = _inputs(dt, sr, m, n, k, 100 + si)
        ref = oracle_mod.tgemm(sr, A, B)
        for var in variants:
            with env(BTAS_CFG=cfg, **var):
                C = host(btas.gemm(dev(A), dev(B), sr))
            np.testing.assert_array_equal(bits(C), bits(ref), err_msg=f"{dt} sr={sr} {m}x{n}x{k} {var} cfg={cfg}")


@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_accumulate_trans_b_and_strided(btas, oracle_mod, dt, sr):
    import torch
    m, n, k = 150, 90, 77
    A, B = _inputs(dt, sr, m, n, k, 7)
    C0 = int_matrix(9, (m, n), sr) if dt == "i32" else f32_matrix(9, (m, n), sr)
    ref_acc = oracle_mod.tgemm(sr, A, B, C0)
    out = dev(C0)
    btas.gemm(dev(A), dev(B), sr, out=out, accumulate=True)
    np.testing.assert_array_equal(bits(host(out)), bits(ref_acc))
    # B given transposed
    ref = oracle_mod.tgemm(sr, A, B)
    C = host(btas.gemm(dev(A), dev(np.ascontiguousarray(B.T)), sr, trans_b=True))
    np.testing.assert_array_equal(bits(C), bits(ref))
    # strided views: lda > k, ldb > n, ldc > n (aligned and unaligned pitch)
    for pad in (4, 3):
        Abig = dev(np.pad(A, ((0, 0), (0, pad))))
        Bbig = dev(np.pad(B, ((0, 0), (0, pad))))
        Cbig = torch.zeros((m, n + pad), dtype=Abig.dtype, device="cuda")
        btas.gemm(Abig[:, :k], Bbig[:, :n], sr, out=Cbig[:, :n])
        np.testing.assert_array_equal(bits(host(Cbig[:, :n]).copy()), bits(ref))
        assert (host(Cbig[:, n:]) == 0).all()  # padding untouched


@pytest.mark.parametrize("sr", [0, 1])
def test_k_zero_writes_identity(btas, sr):
    import torch
    A = torch.empty((5, 0), dtype=torch.int32, device="cuda")
    B = torch.empty((0, 7), dtype=torch.int32, device="cuda")
    C = host(btas.gemm(A, B, sr))
    assert (C == (INF if sr == 0 else NINF)).all()
    Af = torch.empty((5, 0), dtype=torch.float32, device="cuda")
    Bf = torch.empty((0, 7), dtype=torch.float32, device="cuda")
    Cf = host(btas.gemm(Af, Bf, sr))
    assert (Cf == (np.inf if sr == 0 else -np.inf)).all()


def test_identity_and_duality_on_gpu(btas):
    """Semiring laws hold for the kernel's own outputs (sizes spanning tiles)."""
    n = 300
    A = int_matrix(21, (n, n), 0)
    E = np.full((n, n), INF, np.int32)
    np.fill_diagonal(E, 0)
    np.testing.assert_array_equal(host(btas.gemm(dev(E), dev(A), 0)), A)
    np.testing.assert_array_equal(host(btas.gemm(dev(A), dev(E), 0)), A)
    Am = int_matrix(22, (n, 200), 1)
    Bm = int_matrix(23, (200, 170), 1)
    mx = host(btas.gemm(dev(Am), dev(Bm), 1))
    mn = host(btas.gemm(dev(-Am), dev(-Bm), 0))
    np.testing.assert_array_equal(mx, -mn)


@pytest.mark.parametrize("ns", ["0", "4", "5", "8"])
def test_u16_packed_product(btas, oracle_mod, ns):
    import torch
    for (m, n, k) in [(1, 1, 1), (5, 7, 3), (130, 258, 40), (300, 511, 257)]:
        A = gen.uniform_int(31 + m, 1, (m, k), 0, 0x7FFF).astype(np.uint16)
        B = gen.uniform_int(32 + n, 1, (k, n), 0, 0x7FFF).astype(np.uint16)
        ref = oracle_mod.tgemm_u16(A, B)
        with env(BTAS_U16_NS=ns):
            C = btas.gemm(dev(A.view(np.int16)), dev(B.view(np.int16)), 0)
        np.testing.assert_array_equal(host(C).view(np.uint16), ref, err_msg=f"{m}x{n}x{k} ns={ns}")


@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_full_size_8192_sampled_rows(btas, oracle_mod, dt, sr):
    """M = N = K = 8192 in the launch configuration the benchmark times:
    FP32 uniform [0, 1) and int32 uniform [0, 10^6]; 64 seeded full rows are
    recomputed by the oracle."""
    n = 8192
    if dt == "i32":
        A = gen.uniform_int(gen.BASE_SEED, 21, (n, n), 0, 10 ** 6)
        B = gen.uniform_int(gen.BASE_SEED, 22, (n, n), 0, 10 ** 6)
    else:
        A = gen.uniform_f32(gen.BASE_SEED, 23, (n, n))
        B = gen.uniform_f32(gen.BASE_SEED, 24, (n, n))
    C = host(btas.gemm(dev(A), dev(B), sr))
    rows = gen.sample_indices(gen.BASE_SEED, 25, 64, n)
    oracle_mod.set_threads(os.cpu_count() or 1)
    try:
        ref = oracle_mod.tgemm(sr, A[rows], B)
    finally:
        oracle_mod.set_threads(1)
    np.testing.assert_array_equal(bits(C[rows]), bits(ref))


def _ranged(seed, shape, lo, hi, sr, p_inf=0.1):
    return int_matrix(seed, shape, sr, lo=lo, hi=hi, p_inf=p_inf)


@pytest.mark.parametrize("sr", [0, 1])
def test_packed_int32_product(btas, oracle_mod, sr):
    """BTAS_GEMM_PACKED: operands whose finite ranges add up to less than
    0x7FFF run on the packed kernel (the device counter moves) and give the
    oracle's bits, negative values, INF entries, ragged sizes, B transposed
    and the accumulate form included; wider ranges or an out-of-domain entry
    keep the int32 kernel, with the same bits."""
    cases = [((1, 1, 1), (-3, 3), (0, 0)), ((31, 33, 17), (-1000, 1000), (5, 900)),
             ((200, 300, 129), (-9000, 4000), (100, 16000)), ((257, 130, 513), (0, 16383), (0, 16383))]
    for si, ((m, n, k), ra, rb) in enumerate(cases):
        A = _ranged(300 + si, (m, k), *ra, sr)
        B = _ranged(400 + si, (k, n), *rb, sr)
        ref = oracle_mod.tgemm(sr, A, B)
        c0 = btas.btas_packed_products()
        C = host(btas.gemm(dev(A), dev(B), sr, packed=True))
        assert btas.btas_packed_products() == c0 + 1, (m, n, k)
        np.testing.assert_array_equal(C, ref, err_msg=f"{m}x{n}x{k}")
        Ct = host(btas.gemm(dev(A), dev(np.ascontiguousarray(B.T)), sr, trans_b=True, packed=True))
        np.testing.assert_array_equal(Ct, ref)
        C0 = _ranged(500 + si, (m, n), -20000, 20000, sr)
        out = dev(C0)
        btas.gemm(dev(A), dev(B), sr, out=out, accumulate=True, packed=True)
        np.testing.assert_array_equal(host(out), oracle_mod.tgemm(sr, A, B, C0))
        assert btas.btas_packed_products() == c0 + 3
    # ranges too wide (about 20000 + 20000 >= 0x7FFF): int32 kernel, same bits
    A = _ranged(600, (100, 70), 0, 20000, sr)
    B = _ranged(601, (70, 90), -20000, 0, sr)
    c0 = btas.btas_packed_products()
    np.testing.assert_array_equal(host(btas.gemm(dev(A), dev(B), sr, packed=True)), oracle_mod.tgemm(sr, A, B))
    assert btas.btas_packed_products() == c0
    # the other semiring's identity is outside the domain: int32 kernel
    A = _ranged(604, (100, 70), -10, 10, sr)
    A[3, 4] = NINF if sr == 0 else INF
    btas.gemm(dev(A), dev(_ranged(602, (70, 90), 0, 10, sr)), sr, packed=True)
    assert btas.btas_packed_products() == c0
    # all-identity operand: packed, every output is the identity
    E = np.full((40, 30), INF if sr == 0 else NINF, np.int32)
    c0 = btas.btas_packed_products()
    C = host(btas.gemm(dev(E), dev(_ranged(603, (30, 50), -5, 5, sr)), sr, packed=True))
    assert btas.btas_packed_products() == c0 + 1
    assert (C == (INF if sr == 0 else NINF)).all()


def test_packed_strided_operands(btas, oracle_mod):
    """Packed path with leading dimensions larger than the rows (aligned and
    unaligned pitch) on A, B and C."""
    import torch
    m, n, k = 130, 97, 61
    for sr in (0, 1):
        A = _ranged(650 + sr, (m, k), -500, 700, sr)
        B = _ranged(660 + sr, (k, n), 0, 900, sr)
        ref = oracle_mod.tgemm(sr, A, B)
        for pad in (4, 3):
            Ab = dev(np.pad(A, ((0, 0), (0, pad))))
            Bb = dev(np.pad(B, ((0, 0), (0, pad))))
            Cb = torch.zeros((m, n + pad), dtype=torch.int32, device="cuda")
            c0 = btas.btas_packed_products()
            btas.gemm(Ab[:, :k], Bb[:, :n], sr, out=Cb[:, :n], packed=True)
            assert btas.btas_packed_products() == c0 + 1
            np.testing.assert_array_equal(host(Cb[:, :n]).copy(), ref)
            assert (host(Cb[:, n:]) == 0).all()


def test_packed_full_size_sampled_rows(btas, oracle_mod):
    """n = 8192 int32 min-plus with values in [0, 8000]: packed path at full
    size, 32 seeded rows recomputed by the oracle."""
    n = 8192
    A = gen.uniform_int(gen.BASE_SEED, 71, (n, n), 0, 8000)
    B = gen.uniform_int(gen.BASE_SEED, 72, (n, n), 0, 8000)
    c0 = btas.btas_packed_products()
    C = btas.gemm(dev(A), dev(B), 0, packed=True)
    assert btas.btas_packed_products() == c0 + 1
    rows = gen.sample_indices(gen.BASE_SEED, 73, 32, n)
    ref = oracle_mod.tgemm(0, A[rows], B)
    np.testing.assert_array_equal(host(C[torch_index(rows)]), ref)


def torch_index(rows):
    import torch
    return torch.from_numpy(np.asarray(rows, dtype=np.int64)).cuda()


@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_checked_in_domain(btas, oracle_mod, dt, sr):
    """BTAS_GEMM_CHECKED on operands inside the domain (INF entries
    included): the same bits as the oracle, and btas_sync_status reports
    nothing -- plain, accumulate, B transposed and (int32) packed."""
    m, n, k = 200, 150, 90
    A, B = _inputs(dt, sr, m, n, k, 4100 + sr)
    ref = oracle_mod.tgemm(sr, A, B)
    np.testing.assert_array_equal(bits(host(btas.gemm(dev(A), dev(B), sr, checked=True))), bits(ref))
    np.testing.assert_array_equal(
        bits(host(btas.gemm(dev(A), dev(np.ascontiguousarray(B.T)), sr, trans_b=True, checked=True))), bits(ref))
    C0 = _inputs(dt, sr, m, n, 1, 4200 + sr)[0][:, :1].repeat(n, axis=1)
    acc = host(btas.gemm(dev(A), dev(B), sr, out=dev(C0), accumulate=True, checked=True))
    np.testing.assert_array_equal(bits(acc), bits(oracle_mod.tgemm(sr, A, B, C0)))
    if dt == "i32":
        Ap = gen.uniform_int(gen.BASE_SEED, 4300, (m, k), -2000, 2000)
        Bp = gen.uniform_int(gen.BASE_SEED, 4301, (k, n), -2000, 2000)
        np.testing.assert_array_equal(host(btas.gemm(dev(Ap), dev(Bp), sr, packed=True, checked=True)),
                                      oracle_mod.tgemm(sr, Ap, Bp))
    assert btas.sync_status() == (0, 0, 0)


@pytest.mark.parametrize("sr", [0, 1])
@pytest.mark.parametrize("dt", ["i32", "f32"])
def test_checked_out_of_domain(btas, dt, sr):
    """An operand entry outside the domain: the checked product leaves C
    unwritten, the call itself returns BTAS_OK (it stays asynchronous), and
    btas_sync_status reports the entries and calls once, then clears."""
    import torch
    m, n, k = 130, 70, 50
    A, B = _inputs(dt, sr, m, n, k, 4400 + sr)
    A, B = A.copy(), B.copy()
    if dt == "i32":
        A[3, 4] = 1 << 29  # beyond 2^28 and not INF
        B[7, 1] = NINF if sr == 0 else INF  # the other semiring's identity
    else:
        A[3, 4] = np.float32("nan")
        B[7, 1] = np.float32("-inf") if sr == 0 else np.float32("inf")
    sentinel = np.full((m, n), 41, dtype=A.dtype)
    for packed in ((False, True) if dt == "i32" else (False,)):
        out = dev(sentinel)
        btas.gemm(dev(A), dev(B), sr, out=out, packed=packed, checked=True)
        assert btas.sync_status() == (1, 2, 1)
        np.testing.assert_array_equal(host(out), sentinel)
    # accumulate: an out-of-domain entry of C is found too
    good_a, good_b = _inputs(dt, sr, m, n, k, 4500 + sr)
    C0 = np.array(sentinel)
    C0[0, 0] = (1 << 29) if dt == "i32" else np.float32("nan")
    out = dev(C0)
    btas.gemm(dev(good_a), dev(good_b), sr, out=out, accumulate=True, checked=True)
    assert btas.sync_status() == (1, 1, 1)
    np.testing.assert_array_equal(bits(host(out)), bits(C0))
    assert btas.sync_status() == (0, 0, 0)
    torch.cuda.synchronize()


@pytest.mark.parametrize("dt", ["i32", "f32", "u16"])
def test_wave_raster_and_backward_k(btas, oracle_mod, dt):
    """Grids of two or more waves take the column-group raster with k run
    backwards in every other wave: same bits as the oracle and as the
    row-group raster (BTAS_KWAVE=0), at ragged m, n and k (k = 77 and 45 end
    on a partial slice, which a backward wave loads first)."""
    if dt == "u16":
        m, n, k = 4100, 2400, 45
        A = gen.uniform_int(61, 1, (m, k), 0, 0x7FFF).astype(np.uint16)
        B = gen.uniform_int(62, 1, (k, n), 0, 0x7FFF).astype(np.uint16)
        ref = oracle_mod.tgemm_u16(A, B)
        C = host(btas.gemm(dev(A.view(np.int16)), dev(B.view(np.int16)), 0)).view(np.uint16)
        with env(BTAS_KWAVE="0"):
            C0 = host(btas.gemm(dev(A.view(np.int16)), dev(B.view(np.int16)), 0)).view(np.uint16)
    else:
        m, n, k = 3200, 3100, 77
        A, B = _inputs(dt, 0, m, n, k, 63)
        oracle_mod.set_threads(os.cpu_count() or 1)
        try:
            ref = oracle_mod.tgemm(0, A, B)
        finally:
            oracle_mod.set_threads(1)
        C = host(btas.gemm(dev(A), dev(B), 0))
        with env(BTAS_KWAVE="0"):
            C0 = host(btas.gemm(dev(A), dev(B), 0))
        # accumulate into a prior C, B supplied transposed: the same raster
        Cp = (int_matrix(64, (m, n), 0) if dt == "i32" else f32_matrix(64, (m, n), 0))
        oracle_mod.set_threads(os.cpu_count() or 1)
        try:
            ref_acc = oracle_mod.tgemm(0, A, B, Cp)
        finally:
            oracle_mod.set_threads(1)
        acc = dev(Cp)
        btas.gemm(dev(A), dev(np.ascontiguousarray(B.T)), 0, out=acc, accumulate=True, trans_b=True)
        np.testing.assert_array_equal(bits(host(acc)), bits(ref_acc))
    np.testing.assert_array_equal(bits(C), bits(ref))
    np.testing.assert_array_equal(bits(C0), bits(ref))
