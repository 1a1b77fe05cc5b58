"""The kernel autotuner on the GPU: every candidate it times must give the
same bits (it checks this itself), the kernel it picks must reproduce the
oracle, and a table entry -- tuned, loaded from a file, or tuned on the spot
under BTAS_TUNE=1 -- must be what the library then runs, with unchanged
results."""
import json
import os

import numpy as np
import pytest

import gen
from gpu_util import bits, dev, f32_matrix, host, int_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture()
def btas():
    import torch
    import paper_1701_04733_gb300 as b
    assert torch.cuda.is_available()
    b.lib()
    b.tune_clear()
    yield b
    b.tune_clear()


class env:
    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        self.old = {k: os.environ.get(k) for k in self.kv}
        for k, v in self.kv.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v

    def __exit__(self, *a):
        for k, v in self.old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def _pair(dt, sr, m, n, k, seed):
    if dt == "i32":
        return int_matrix(seed, (m, k), sr), int_matrix(seed + 1, (k, n), sr)
    return f32_matrix(seed, (m, k), sr), f32_matrix(seed + 1, (k, n), sr)


@pytest.mark.parametrize("sr,dt", [(0, "i32"), (1, "i32"), (0, "f32"), (1, "f32")])
def test_tune_then_gemm_matches_oracle(btas, oracle_mod, sr, dt):
    code = btas.I32 if dt == "i32" else btas.F32
    m, n, k = 300, 260, 150
    r = btas.tune_gemm(sr, code, m, n, k)
    assert r["candidates"] >= 3 and r["seconds"] > 0 and r["terms_per_second"] > 0
    assert r["group_m"] in (1, 4, 8, 16) and r["tile_m"] in (64, 128)
    assert (r["variant"] in (0, 1)) == (dt == "i32")
    assert btas.tune_lookup(sr, code, m, n, k) == r
    # the same size buckets share the entry; another bucket has none
    assert btas.tune_lookup(sr, code, 257, 511, 129) == r
    assert btas.tune_lookup(sr, code, 600, 260, 150) is None
    A, B = _pair(dt, sr, m, n, k, 40 + sr)
    ref = oracle_mod.tgemm(sr, A, B)
    np.testing.assert_array_equal(bits(host(btas.gemm(dev(A), dev(B), sr))), bits(ref))


def test_tune_u16_then_packed_product(btas, oracle_mod):
    m, n, k = 200, 300, 130
    r = btas.tune_gemm(0, btas.U16, m, n, k)
    assert r["variant"] == btas.TUNE_VARIANT_U16 and r["ns"] in (0, 4, 5, 6, 8) and r["candidates"] == 5
    A = gen.uniform_int(51, 1, (m, k), 0, 0x7FFF).astype(np.uint16)
    B = gen.uniform_int(52, 1, (k, n), 0, 0x7FFF).astype(np.uint16)
    C = btas.gemm(dev(A.view(np.int16)), dev(B.view(np.int16)), 0)
    np.testing.assert_array_equal(host(C).view(np.uint16), oracle_mod.tgemm_u16(A, B))


def _entry(sr, dt, m, n, k, **kv):
    import torch
    p = torch.cuda.get_device_properties(0)
    b = lambda x: int(np.ceil(np.log2(x))) if x > 1 else 0
    e = {"arch": p.major * 10 + p.minor, "sms": p.multi_processor_count, "semiring": sr, "dtype": dt,
         "m_bucket": b(m), "n_bucket": b(n), "k_bucket": b(k), "variant": 0, "ns": 0, "cfg": 0, "group_m": 8,
         "candidates": 1, "tile_m": 128, "tile_n": 128, "seconds": 1.0, "terms_per_second": 1.0}
    e.update(kv)
    return json.dumps(e)


@pytest.mark.parametrize("entry", [
    dict(variant=0, ns=0, cfg=2, group_m=3, tile_m=64, tile_n=64),   # DPX, 64 x 64 tiles, odd raster group
    dict(variant=1, ns=8, cfg=0, group_m=1),                         # mixed, all columns on IMAD, no grouping
    dict(variant=1, ns=5, cfg=5, group_m=16),                        # 2 CTAs/SM, 128-bit fragments
])
def test_loaded_entry_is_used_and_exact(btas, oracle_mod, tmp_path, entry):
    """A table entry naming a non-default kernel and raster group routes the
    product (and the APSP squarings of the same buckets) through it."""
    m = n = k = 333
    p = tmp_path / "t.jsonl"
    p.write_text(_entry(0, btas.I32, m, n, k, **entry) + "\n")
    assert btas.tune_load(str(p)) == 1
    assert btas.tune_lookup(0, btas.I32, m, n, k)["cfg"] == entry["cfg"]
    A, B = _pair("i32", 0, m, n, k, 60)
    np.testing.assert_array_equal(host(btas.gemm(dev(A), dev(B), 0)), oracle_mod.tgemm(0, A, B))
    # weights above 2^23: every squaring runs on the int32 kernels
    W = gen.random_graph(61, 0, n, 0.05, 1, 2 * 10**7)
    D, info = btas.apsp(dev(W), info=True)
    assert set(info["path"].split("+")) - {"sparse"} == {"int32"}
    np.testing.assert_array_equal(host(D), oracle_mod.apsp_squaring(W))


def test_save_clear_load(btas, tmp_path):
    r = btas.tune_gemm(1, btas.F32, 130, 140, 150)
    p = tmp_path / "cache.jsonl"
    btas.tune_save(str(p))
    btas.tune_clear()
    assert btas.tune_lookup(1, btas.F32, 130, 140, 150) is None
    assert btas.tune_load(str(p)) == 1
    got = btas.tune_lookup(1, btas.F32, 130, 140, 150)
    assert {k: got[k] for k in ("variant", "ns", "cfg", "group_m", "tile_m", "tile_n", "candidates")} == \
        {k: r[k] for k in ("variant", "ns", "cfg", "group_m", "tile_m", "tile_n", "candidates")}
    assert got["seconds"] == pytest.approx(r["seconds"], rel=1e-8)


def test_on_the_spot_tuning(btas, oracle_mod, tmp_path):
    """BTAS_TUNE=1: the first product of an untuned bucket tunes it (and
    appends the table to BTAS_TUNE_CACHE); the result is still exact."""
    cache = tmp_path / "spot.jsonl"
    m, n, k = 90, 500, 70
    A, B = _pair("f32", 0, m, n, k, 70)
    with env(BTAS_TUNE="1", BTAS_TUNE_CACHE=str(cache)):
        C = host(btas.gemm(dev(A), dev(B), 0))
    np.testing.assert_array_equal(bits(C), bits(oracle_mod.tgemm(0, A, B)))
    assert btas.tune_entries() == 1
    assert btas.tune_lookup(0, btas.F32, m, n, k) is not None
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and json.loads(lines[0])["dtype"] == btas.F32
    # without BTAS_TUNE a new bucket stays untuned
    with env(BTAS_TUNE=None):
        btas.gemm(dev(A[:, :20]), dev(B[:20]), 0)
    assert btas.tune_entries() == 1


def test_env_override_beats_table(btas, oracle_mod, tmp_path):
    m = n = k = 200
    p = tmp_path / "t.jsonl"
    p.write_text(_entry(1, btas.I32, m, n, k, variant=1, ns=4, cfg=4) + "\n")
    btas.tune_load(str(p))
    A, B = _pair("i32", 1, m, n, k, 80)
    with env(BTAS_CFG="0", BTAS_I32_VARIANT="0"):
        C = host(btas.gemm(dev(A), dev(B), 1))
    np.testing.assert_array_equal(C, oracle_mod.tgemm(1, A, B))
