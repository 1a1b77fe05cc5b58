"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/btas.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(btas_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    import paper_1701_04733_gb300 as btas
    return btas.build()


def test_header_declares_core_calls():
    names = _declared()
    for must in ("btas_gemm", "btas_dot", "btas_axpy", "btas_add", "btas_mul", "btas_apsp", "btas_apsp_ex",
                 "btas_last_error_string"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    import paper_1701_04733_gb300 as btas
    assert set(_declared()) <= set(btas.SIGNATURES), set(_declared()) - set(btas.SIGNATURES)
    btas.lib()  # loads and binds every signature


def test_host_side_argument_errors(libpath):
    """Argument checks run on the host before anything touches a GPU."""
    import paper_1701_04733_gb300 as btas
    assert btas.btas_version() >= 100
    # negative size
    assert btas.btas_gemm(0, 0, -1, 4, 4, None, 4, None, 4, None, 4, None) == 1
    # unknown semiring / dtype / flag bits
    assert btas.btas_gemm(7, 0, 4, 4, 4, None, 4, None, 4, None, 4, None) == 1
    assert btas.btas_gemm(0, 9, 4, 4, 4, None, 4, None, 4, None, 4, None) == 1
    assert btas.btas_gemm(0x8000, 0, 4, 4, 4, None, 4, None, 4, None, 4, None) == 1
    # short leading dimension
    assert btas.btas_gemm(0, 0, 4, 4, 8, None, 4, None, 4, None, 4, None) == 1
    assert "lda" in btas.last_error()
    # max-plus on the 16-bit path is not offered
    assert btas.btas_gemm(1, 2, 4, 4, 4, 1, 4, 1, 4, 1, 4, None) == 7
    # the issue-rate probe: mixes 0..15 at 1 or 2 CTAs per SM
    assert btas.btas_measure_issue_rate_ex(16, 1, None) == 1
    assert btas.btas_measure_issue_rate_ex(0, 3, None) == 1
    assert btas.btas_measure_issue_rate(8, None) == 1  # the diagnostic mixes need the _ex form
    # the batched launch's tile tuner takes 1 <= n_max <= 2048
    assert btas.btas_batch_tune(0, None, None, 0) == 1
    assert btas.btas_batch_tune(4096, None, None, 0) == 1
    # the domain check covers int32 and fp32 only
    assert btas.btas_gemm(0x1000, 2, 4, 4, 4, 1, 4, 1, 4, 1, 4, None) == 7
    assert "CHECKED" in btas.last_error()
    # empty problems are no-ops
    assert btas.btas_gemm(0, 0, 0, 4, 4, None, 4, None, 4, None, 4, None) == 0
    assert btas.btas_apsp(0, None, None, None) == 0
    assert btas.btas_apsp(-3, None, None, None) == 1
    assert btas.btas_apsp_ex(4, 1, 1, 0x6, None, None, None, None) == 1  # two FORCE flags
    assert btas.btas_apsp_u16(100, 1, 1, 400, 0, None) == 2  # 99*400 >= 0x7FFF
    assert btas.btas_dot(0, 0, 10, 1, 0, 1, 1, 1, None) == 1  # zero stride
    assert btas.btas_apsp_squarings(256) == 8 and btas.btas_apsp_squarings(8192) == 13
