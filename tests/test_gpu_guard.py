"""Out-of-bounds write checks (a stand-in for a memory sanitizer): every
output and input of every entry point sits inside a larger device (or host)
allocation whose 4 KiB guard bands before and after hold a fill pattern; the
call must leave both bands, and every input, bit-for-bit unchanged, and the
result must still match the oracle.  Sizes are ragged (not multiples of the
tile sizes or of 4)."""
import numpy as np
import pytest

import gen
from gpu_util import bits, f32_matrix, host, int_matrix

pytestmark = pytest.mark.gpu

GUARD = 4096   # bytes on each side
FILL = 0xA5


class Guarded:
    """A tensor of `shape` placed in the middle of a guard-banded buffer."""

    def __init__(self, init, device="cuda"):
        import torch
        t = torch.from_numpy(np.ascontiguousarray(init))
        nb = t.numel() * t.element_size()
        self.raw = torch.full((2 * GUARD + nb,), FILL, dtype=torch.uint8, device=device)
        if device == "cpu":
            self.raw = self.raw.pin_memory()
        self.t = self.raw[GUARD:GUARD + nb].view(t.dtype).view(t.shape)
        self.t.copy_(t)
        self.init = np.ascontiguousarray(init).copy()
        self.nb = nb

    def guards_intact(self):
        r = self.raw.cpu().numpy()
        return bool((r[:GUARD] == FILL).all() and (r[GUARD + self.nb:] == FILL).all())

    def unchanged(self):
        return np.array_equal(bits(host(self.t)), bits(self.init))


@pytest.fixture(scope="module")
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    return b


def _out(shape, dtype):
    return Guarded(np.zeros(shape, dtype))


def _check(*gs):
    for g in gs:
        assert g.guards_intact(), "a guard band was overwritten"


@pytest.mark.parametrize("dt", ["i32", "f32", "u16"])
@pytest.mark.parametrize("sr", [0, 1])
def test_gemm(btas, oracle_mod, dt, sr):
    if dt == "u16" and sr == 1:
        pytest.skip("packed 16-bit is min-plus only")
    m, n, k = 130, 257, 75
    if dt == "u16":
        A = gen.uniform_int(11, 1, (m, k), 0, 0x7FFF).astype(np.uint16).view(np.int16)
        B = gen.uniform_int(12, 1, (k, n), 0, 0x7FFF).astype(np.uint16).view(np.int16)
        ref = oracle_mod.tgemm_u16(A.view(np.uint16), B.view(np.uint16)).view(np.int16)
    else:
        mk = int_matrix if dt == "i32" else f32_matrix
        A, B = mk(11, (m, k), sr), mk(12, (k, n), sr)
        ref = oracle_mod.tgemm(sr, A, B)
    gA, gB, gC = Guarded(A), Guarded(B), _out((m, n), ref.dtype)
    btas.gemm(gA.t, gB.t, sr, out=gC.t)
    _check(gA, gB, gC)
    assert gA.unchanged() and gB.unchanged()
    np.testing.assert_array_equal(bits(host(gC.t)), bits(ref))
    if dt == "i32":
        # exact packed path (small-range operands), plain and B transposed
        Ap, Bp = int_matrix(13, (m, k), sr, -2000, 2000), int_matrix(14, (k, n), sr, -2000, 2000)
        refp = oracle_mod.tgemm(sr, Ap, Bp)
        gAp, gBp, gBpt, gCp = Guarded(Ap), Guarded(Bp), Guarded(np.ascontiguousarray(Bp.T)), _out((m, n), np.int32)
        c0 = btas.btas_packed_products()
        btas.gemm(gAp.t, gBp.t, sr, out=gCp.t, packed=True)
        _check(gAp, gBp, gCp)
        np.testing.assert_array_equal(host(gCp.t), refp)
        btas.gemm(gAp.t, gBpt.t, sr, out=gCp.t, packed=True, trans_b=True)
        _check(gBpt, gCp)
        np.testing.assert_array_equal(host(gCp.t), refp)
        assert btas.btas_packed_products() == c0 + 2
    if dt != "u16":
        gBt = Guarded(np.ascontiguousarray(B.T))
        gC2 = Guarded(ref)  # accumulate into the result itself: unchanged (idempotent)
        btas.gemm(gA.t, gBt.t, sr, out=gC2.t, accumulate=True, trans_b=True)
        _check(gBt, gC2)
        np.testing.assert_array_equal(bits(host(gC2.t)), bits(ref))


@pytest.mark.parametrize("flags", ["default", "i32", "carrier", "u16"])
def test_apsp_modes(btas, oracle_mod, flags):
    n = 301
    whi = 20 if flags == "u16" else 1000
    W = gen.random_graph(21, 1, n, 0.05, 1, whi)
    ref = oracle_mod.apsp_squaring(W)
    f = {"default": btas.APSP_EARLY_EXIT, "i32": btas.APSP_EARLY_EXIT | btas.APSP_FORCE_I32,
         "carrier": btas.APSP_EARLY_EXIT | btas.APSP_FORCE_CARRIER,
         "u16": btas.APSP_EARLY_EXIT | btas.APSP_FORCE_U16}[flags]
    gW, gD = Guarded(W), _out((n, n), np.int32)
    btas.apsp(gW.t, out=gD.t, flags=f)
    _check(gW, gD)
    assert gW.unchanged()
    np.testing.assert_array_equal(host(gD.t), ref)


def test_apsp_u16_storage_paths_fw_noalloc(btas, oracle_mod):
    import torch
    n = 203
    W = gen.random_graph(22, 1, n, 0.05, 1, 30)
    ref = oracle_mod.apsp_squaring(W)
    # 16-bit storage
    W16 = np.where(W >= 0x7FFF, 0x7FFF, W).astype(np.uint16).view(np.int16)
    gW16, gD16 = Guarded(W16), _out((n, n), np.int16)
    btas.apsp_u16(gW16.t, 30, out=gD16.t)
    _check(gW16, gD16)
    assert gW16.unchanged()
    np.testing.assert_array_equal(np.minimum(host(gD16.t).view(np.uint16).astype(np.int64), 0x7FFF),
                                  np.where(ref >= 0x7FFF, 0x7FFF, ref))
    # next-hop matrix
    gW = Guarded(W)
    D, Nx = btas.apsp_paths(gW.t)
    assert gW.unchanged() and gW.guards_intact()
    # paths into guarded outputs through the raw binding
    gD, gN = _out((n, n), np.int32), _out((n, n), np.int32)
    st = torch.cuda.current_stream().cuda_stream
    btas.check(btas.btas_apsp_paths(n, gW.t.data_ptr(), gD.t.data_ptr(), gN.t.data_ptr(), btas.APSP_EARLY_EXIT,
                                    None, st))
    _check(gD, gN)
    np.testing.assert_array_equal(host(gD.t), ref)
    np.testing.assert_array_equal(host(gN.t), host(Nx))
    # binary32 next-hop matrix into guarded outputs
    Wf = np.where(W >= 0x3FFFFFFF, np.float32(np.inf), W.astype(np.float32)).astype(np.float32)
    gWf, gDf, gNf = Guarded(Wf), _out((n, n), np.float32), _out((n, n), np.int32)
    btas.check(btas.btas_apsp_paths_f32(n, gWf.t.data_ptr(), gDf.t.data_ptr(), gNf.t.data_ptr(),
                                        btas.APSP_EARLY_EXIT, None, st))
    _check(gWf, gDf, gNf)
    assert gWf.unchanged()
    np.testing.assert_array_equal(host(gDf.t), np.where(ref >= 0x3FFFFFFF, np.float32(np.inf), ref.astype(np.float32)))
    np.testing.assert_array_equal(host(gNf.t), host(Nx))
    # blocked Floyd-Warshall
    gF = _out((n, n), np.int32)
    btas.apsp_fw(gW.t, out=gF.t)
    _check(gW, gF)
    np.testing.assert_array_equal(host(gF.t), ref)
    # allocation-free entry point
    gA = _out((n, n), np.int32)
    btas.check(btas.btas_apsp_noalloc(n, gW.t.data_ptr(), gA.t.data_ptr(), st))
    torch.cuda.synchronize()
    _check(gW, gA)
    np.testing.assert_array_equal(host(gA.t), ref)


@pytest.mark.parametrize("dt", ["i32", "f32"])
@pytest.mark.parametrize("sr", [0, 1])
def test_closure(btas, oracle_mod, dt, sr):
    n = 150
    if dt == "i32":
        A = gen.random_graph(23, 1, n, 0.05, 1, 50)
        if sr == 1:
            A = np.where(A == gen.INF_I32, -gen.INF_I32, -A).astype(np.int32)
    else:
        A = np.full((n, n), np.inf if sr == 0 else -np.inf, np.float32)
        mask = gen.uniform_unit_f64(24, 1, np.arange(n * n, dtype=np.uint64)).reshape(n, n) < 0.05
        vals = gen.uniform_f32(24, 2, (n, n)) * np.float32(8.0)
        A[mask] = vals[mask] if sr == 0 else -vals[mask]
        np.fill_diagonal(A, np.float32(0.0))
    gA, gS = Guarded(A), _out((n, n), A.dtype)
    btas.closure(gA.t, sr, out=gS.t)
    _check(gA, gS)
    assert gA.unchanged()
    ref = oracle_mod.apsp_squaring(A) if (dt == "i32" and sr == 0) else None
    if ref is not None:
        np.testing.assert_array_equal(host(gS.t), ref)


def test_gemv_sssp_and_vector_ops(btas, oracle_mod):
    m, n = 301, 257
    for sr in (0, 1):
        A = int_matrix(31, (m, n), sr)
        x = int_matrix(32, (1, n), sr)[0]
        xt = int_matrix(33, (1, m), sr)[0]
        gA, gx, gxt = Guarded(A), Guarded(x), Guarded(xt)
        gy, gyt = _out((m,), np.int32), _out((n,), np.int32)
        btas.gemv(gA.t, gx.t, sr, out=gy.t)
        btas.gemv(gA.t, gxt.t, sr, trans=True, out=gyt.t)
        _check(gA, gx, gxt, gy, gyt)
        np.testing.assert_array_equal(host(gy.t), oracle_mod.gemv(sr, A, x))
        np.testing.assert_array_equal(host(gyt.t), oracle_mod.gemv(sr, A, xt, trans=True))
        # level 1
        u = int_matrix(34, (1, 1001), sr)[0]
        v = int_matrix(35, (1, 1001), sr)[0]
        gu, gv, gz, gd = Guarded(u), Guarded(v), _out((1001,), np.int32), _out((), np.int32)
        btas.add(gu.t, gv.t, sr, out=gz.t)
        _check(gu, gv, gz)
        np.testing.assert_array_equal(host(gz.t), oracle_mod.add(sr, u, v))
        btas.mul(gu.t, gv.t, sr, out=gz.t)
        _check(gz)
        np.testing.assert_array_equal(host(gz.t), oracle_mod.mul(sr, u, v))
        btas.dot(gu.t, gv.t, sr, out=gd.t)
        _check(gd)
        assert int(host(gd.t).reshape(-1)[0]) == int(oracle_mod.dot(sr, u, v))
        btas.axpy(7, gu.t, gv.t, sr)
        _check(gu, gv)
        np.testing.assert_array_equal(host(gv.t), oracle_mod.axpy(sr, 7, u, v))
    W = gen.random_graph(36, 1, 401, 0.02, 1, 100)
    gW = Guarded(W)
    d = btas.sssp(gW.t, 5)
    _check(gW)
    np.testing.assert_array_equal(host(d), oracle_mod.sssp(W, 5)[0])


def test_batch_outputs(btas, oracle_mod):
    import torch
    b = btas.Batch()
    cases = []
    for i, n in enumerate((3, 77, 130, 259)):
        W = gen.random_graph(41 + i, 1, n, 0.1, 1, 100)
        gW, gD = Guarded(W), _out((n, n), np.int32)
        b.add_apsp(gW.t, gD.t)
        cases.append(("apsp", W, gW, gD))
    for i, (m, n, k) in enumerate(((5, 131, 9), (130, 129, 257))):
        A, B = f32_matrix(51 + i, (m, k), 1), f32_matrix(52 + i, (k, n), 1)
        gA, gB, gC = Guarded(A), Guarded(B), _out((m, n), np.float32)
        b.add_gemm(gA.t, gB.t, gC.t, 1)
        cases.append(("gemm", (A, B), (gA, gB), gC))
    b.launch()
    b.wait()
    torch.cuda.synchronize()
    for kind, inp, gin, gout in cases:
        if kind == "apsp":
            _check(gin, gout)
            assert gin.unchanged()
            np.testing.assert_array_equal(host(gout.t), oracle_mod.apsp_squaring(inp))
        else:
            _check(*gin, gout)
            np.testing.assert_array_equal(bits(host(gout.t)), bits(oracle_mod.tgemm(1, *inp)))
    b.close()


def test_server_host_buffers(btas, oracle_mod):
    s = btas.Server(1 << 30)
    W = gen.random_graph(61, 1, 211, 0.05, 1, 100)
    A, B = int_matrix(62, (99, 131), 0), int_matrix(63, (131, 77), 0)
    gW, gD = Guarded(W, "cpu"), Guarded(np.zeros_like(W), "cpu")
    gA, gB, gC = Guarded(A, "cpu"), Guarded(B, "cpu"), Guarded(np.zeros((99, 77), np.int32), "cpu")
    s.submit_apsp(gW.t, gD.t)
    s.submit_gemm(gA.t, gB.t, gC.t, 0)
    s.wait_all()
    s.close()
    _check(gW, gD, gA, gB, gC)
    np.testing.assert_array_equal(gD.t.numpy(), oracle_mod.apsp_squaring(W))
    np.testing.assert_array_equal(gC.t.numpy(), oracle_mod.tgemm(0, A, B))
