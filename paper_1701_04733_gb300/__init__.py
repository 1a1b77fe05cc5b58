"""Python binding of the GB300 tropical-algebra library (C ABI in include/btas.h).

The `btas_*` functions are one-to-one ctypes bindings of the C entry points
(argument marshalling only; every step runs in the CUDA kernels of
libbtas.so).  The lower-case helpers (`gemm`, `apsp`, `dot`, ...) take torch
tensors, pass their device pointers and the current CUDA stream, and raise
`BtasError` on a non-zero status.  PyTorch only provides device memory and
streams.

Semirings (Sec. I): MINPLUS, x (+) y = min(x, y), x (.) y = x + y (Eq. 3-4);
MAXPLUS, x (+) y = max(x, y), x (.) y = x + y (Eq. 1-2).
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbtas.so")

MINPLUS = 0
MAXPLUS = 1
GEMM_ACCUMULATE = 0x100
GEMM_TRANS_B = 0x200
GEMM_NO_CARRIER = 0x400
GEMM_PACKED = 0x800
GEMM_CHECKED = 0x1000
I32 = 0
F32 = 1
U16 = 2
APSP_EARLY_EXIT = 0x1
APSP_FORCE_I32 = 0x2
APSP_FORCE_U16 = 0x4
APSP_FORCE_CARRIER = 0x8
INF_I32 = 0x3FFFFFFF
NINF_I32 = -0x3FFFFFFF
I32_FINITE_MAX = 1 << 28
INF_U16 = 0x7FFF

STATUS = {0: "BTAS_OK", 1: "BTAS_ERR_ARG", 2: "BTAS_ERR_BOUND", 3: "BTAS_ERR_NOMEM", 4: "BTAS_ERR_CUDA",
          5: "BTAS_ERR_TIMEOUT", 6: "BTAS_ERR_BUDGET", 7: "BTAS_ERR_UNSUPPORTED", 8: "BTAS_ERR_INTERNAL"}
TUNE_VARIANT_U16 = 16
BATCH_PROFILE = 0x2
BATCH_PROFILE_SLOTS = 12
BATCH_SLOT_NAMES = ("transpose", "copy", "apsp_u16", "apsp_i32", "apsp_done", "gemm_i32", "gemm_f32",
                    "square_u16", "square_i32", "wait", "lists", "cert")


class BtasError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None

_i64, _i32, _vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
# name -> (restype, argtypes); mirrors include/btas.h
SIGNATURES = {
    "btas_version": (_i32, []),
    "btas_last_error_string": (ctypes.c_char_p, []),
    "btas_kernel_launches": (_i64, []),
    "btas_workspace_reserved": (_i64, []),
    "btas_workspace_trim": (_i32, []),
    "btas_measure_issue_rate": (_i32, [_i32, _vp]),
    "btas_measure_issue_rate_ex": (_i32, [_i32, _i32, _vp]),
    "btas_gemm": (_i32, [_i32, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "btas_sync_status": (_i32, [_vp, _vp, _vp]),
    "btas_packed_products": (_i64, []),
    "btas_dot": (_i32, [_i32, _i32, _i64, _vp, _i64, _vp, _i64, _vp, _vp]),
    "btas_axpy": (_i32, [_i32, _i32, _i64, _vp, _vp, _i64, _vp, _i64, _vp]),
    "btas_add": (_i32, [_i32, _i32, _i64, _vp, _vp, _vp, _vp]),
    "btas_mul": (_i32, [_i32, _i32, _i64, _vp, _vp, _vp, _vp]),
    "btas_apsp": (_i32, [_i64, _vp, _vp, _vp]),
    "btas_apsp_ex": (_i32, [_i64, _vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "btas_apsp_u16": (_i32, [_i64, _vp, _vp, _i32, _i32, _vp]),
    "btas_apsp_squarings": (_i32, [_i64]),
    "btas_closure": (_i32, [_i32, _i32, _i64, _vp, _vp, _i32, _vp, _vp]),
    "btas_apsp_paths": (_i32, [_i64, _vp, _vp, _vp, _i32, _vp, _vp]),
    "btas_apsp_paths_f32": (_i32, [_i64, _vp, _vp, _vp, _i32, _vp, _vp]),
    "btas_gemv": (_i32, [_i32, _i32, _i32, _i64, _i64, _vp, _i64, _vp, _vp, _vp]),
    "btas_apsp_fw": (_i32, [_i64, _vp, _vp, _vp]),
    "btas_sssp": (_i32, [_i64, _vp, _i64, _vp, _vp, _vp]),
    "btas_apsp_noalloc": (_i32, [_i64, _vp, _vp, _vp]),
    "btas_apsp_noalloc_status": (_i32, [_vp, _vp]),
    "btas_batch_create": (_i32, [_vp, _i32]),
    "btas_batch_add_apsp": (_i32, [_vp, _i64, _vp, _vp]),
    "btas_batch_add_gemm": (_i32, [_vp, _i32, _i32, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64]),
    "btas_batch_launch": (_i32, [_vp, _vp]),
    "btas_batch_wait": (_i32, [_vp, _vp]),
    "btas_batch_destroy": (_i32, [_vp]),
    "btas_batch_workspace_bytes": (_i64, [_vp]),
    "btas_batch_tasks": (_i32, [_vp]),
    "btas_batch_profile": (_i32, [_vp, _vp, _vp, _i32]),
    "btas_batch_tune": (_i32, [_i64, _vp, _vp, _i32]),
    "btas_batch_tile": (_i32, [_i32, _i64]),
    "btas_batch_tune_clear": (None, []),
    "btas_batch_select_tiles": (_i32, [_vp, _vp, _vp, _vp]),
    "btas_server_create": (_i32, [_vp, _i64, _i32]),
    "btas_server_submit_apsp": (_i32, [_vp, _i64, _vp, _vp, _vp]),
    "btas_server_submit_gemm": (_i32, [_vp, _i32, _i32, _i64, _i64, _i64, _vp, _vp, _vp, _vp]),
    "btas_server_poll": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "btas_server_wait_all": (_i32, [_vp, ctypes.c_double]),
    "btas_server_stats": (_i32, [_vp, _vp, _vp, _vp, _vp]),
    "btas_server_destroy": (_i32, [_vp]),
    "btas_tune_gemm": (_i32, [_i32, _i32, _i64, _i64, _i64, _vp, _vp]),
    "btas_tune_lookup": (_i32, [_i32, _i32, _i64, _i64, _i64, _vp]),
    "btas_tune_save": (_i32, [ctypes.c_char_p]),
    "btas_tune_load": (_i32, [ctypes.c_char_p, _vp]),
    "btas_tune_clear": (None, []),
    "btas_tune_entries": (_i32, []),
}


class TuneResult(ctypes.Structure):
    """btas_tune_result (include/btas.h)."""
    _fields_ = [("variant", ctypes.c_int), ("ns", ctypes.c_int), ("cfg", ctypes.c_int), ("tile_m", ctypes.c_int),
                ("tile_n", ctypes.c_int), ("group_m", ctypes.c_int), ("candidates", ctypes.c_int),
                ("seconds", ctypes.c_double), ("terms_per_second", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    """The loaded libbtas.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; "
                                   "g.build()'` (nvcc, sm_103a); the library has no CPU fallback")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(handle, name)
                f.restype = res
                f.argtypes = args
            _lib = handle
        return _lib


def build(verbose: bool = False) -> str:
    from . import _build
    return _build.build(verbose=verbose)


def last_error() -> str:
    return lib().btas_last_error_string().decode()


def check(status: int) -> None:
    if status != 0:
        raise BtasError(status, last_error())


# ---------------------------------------------------------------- raw ABI
def btas_workspace_reserved() -> int:
    """Bytes the library's workspace pool of the current device holds."""
    return lib().btas_workspace_reserved()


def btas_workspace_trim() -> int:
    """Release the cached workspace of the current device (syncs)."""
    return lib().btas_workspace_trim()


def btas_packed_products() -> int:
    """Products the current device computed on the packed path (syncs)."""
    return lib().btas_packed_products()


def btas_version() -> int:
    return lib().btas_version()


def btas_kernel_launches() -> int:
    return lib().btas_kernel_launches()


def btas_measure_issue_rate(mix, out_ptr) -> int:
    return lib().btas_measure_issue_rate(mix, out_ptr)


def measure_issue_rate(mix: int, ctas_per_sm: int = 1) -> float:
    """Terms per clock per SM of instruction mix `mix` (see btas.h)."""
    v = ctypes.c_double()
    check(btas_measure_issue_rate_ex(mix, ctas_per_sm, ctypes.addressof(v)))
    return v.value


def btas_measure_issue_rate_ex(mix, ctas_per_sm, out_ptr) -> int:
    return lib().btas_measure_issue_rate_ex(mix, ctas_per_sm, out_ptr)


def btas_gemm(semiring, dtype, m, n, k, A, lda, B, ldb, C, ldc, stream) -> int:
    return lib().btas_gemm(semiring, dtype, m, n, k, A, lda, B, ldb, C, ldc, stream)


def btas_dot(semiring, dtype, n, x, incx, y, incy, result, stream) -> int:
    return lib().btas_dot(semiring, dtype, n, x, incx, y, incy, result, stream)


def btas_axpy(semiring, dtype, n, alpha_host_ptr, x, incx, y, incy, stream) -> int:
    return lib().btas_axpy(semiring, dtype, n, alpha_host_ptr, x, incx, y, incy, stream)


def btas_add(semiring, dtype, n, x, y, z, stream) -> int:
    return lib().btas_add(semiring, dtype, n, x, y, z, stream)


def btas_mul(semiring, dtype, n, x, y, z, stream) -> int:
    return lib().btas_mul(semiring, dtype, n, x, y, z, stream)


def btas_apsp(n, W, D, stream) -> int:
    return lib().btas_apsp(n, W, D, stream)


def btas_apsp_ex(n, W, D, flags, squarings_done_ptr, bound_ptr, path_ptr, stream) -> int:
    return lib().btas_apsp_ex(n, W, D, flags, squarings_done_ptr, bound_ptr, path_ptr, stream)


def btas_apsp_u16(n, W, D, max_w, flags, stream) -> int:
    return lib().btas_apsp_u16(n, W, D, max_w, flags, stream)


def btas_apsp_squarings(n) -> int:
    return lib().btas_apsp_squarings(n)


def btas_closure(semiring, dtype, n, A, Astar, flags, squarings_done_ptr, stream) -> int:
    return lib().btas_closure(semiring, dtype, n, A, Astar, flags, squarings_done_ptr, stream)


def closure(A, semiring="min", out=None, early_exit=True, stream=None, info=False):
    """Tropical closure A* = E (+) A (+) A^2 (+) ... of a square int32/fp32
    CUDA matrix by repeated squaring; raises BtasError if a negative
    (min-plus) / positive (max-plus) cycle makes it diverge."""
    torch = _torch()
    n = A.shape[0]
    if A.shape != (n, n) or not A.is_contiguous():
        raise ValueError("A must be a contiguous square matrix")
    if out is None:
        out = torch.empty_like(A)
    sq = ctypes.c_int(0)
    check(btas_closure(_sr(semiring), _dtype_code(A), n, A.data_ptr(), out.data_ptr(),
                       APSP_EARLY_EXIT if early_exit else 0, ctypes.addressof(sq), _stream(stream)))
    return (out, {"squarings": sq.value}) if info else out


def btas_apsp_paths(n, W, D, Next, flags, squarings_done_ptr, stream) -> int:
    return lib().btas_apsp_paths(n, W, D, Next, flags, squarings_done_ptr, stream)


def btas_apsp_paths_f32(n, W, D, Next, flags, squarings_ptr, stream) -> int:
    return lib().btas_apsp_paths_f32(n, W, D, Next, flags, squarings_ptr, stream)


def apsp_paths(W, early_exit=True, stream=None, info=False):
    """APSP distances and next-hop matrix of an int32 or float32 CUDA matrix
    (the next-hop matrix is int32); with info=True also {"squarings":
    squarings that changed D or Next}."""
    torch = _torch()
    n = W.shape[0]
    if W.shape != (n, n) or not W.is_contiguous():
        raise ValueError("W must be a contiguous n x n tensor")
    D = torch.empty_like(W)
    Nx = torch.empty((n, n), dtype=torch.int32, device=W.device)
    sq = ctypes.c_int(0)
    fn = btas_apsp_paths_f32 if W.dtype == torch.float32 else btas_apsp_paths
    check(fn(n, W.data_ptr(), D.data_ptr(), Nx.data_ptr(), APSP_EARLY_EXIT if early_exit else 0,
             ctypes.addressof(sq), _stream(stream)))
    return (D, Nx, {"squarings": sq.value}) if info else (D, Nx)


def btas_apsp_fw(n, W, D, stream) -> int:
    return lib().btas_apsp_fw(n, W, D, stream)


def apsp_fw(W, out=None, stream=None):
    """APSP by blocked Floyd-Warshall (int32 CUDA matrix; out may be W)."""
    torch = _torch()
    n = W.shape[0]
    out = torch.empty_like(W) if out is None else out
    check(btas_apsp_fw(n, W.data_ptr(), out.data_ptr(), _stream(stream)))
    return out


def btas_gemv(semiring, dtype, trans, m, n, A, lda, x, y, stream) -> int:
    return lib().btas_gemv(semiring, dtype, trans, m, n, A, lda, x, y, stream)


def btas_sssp(n, W, src, dist, iterations_ptr, stream) -> int:
    return lib().btas_sssp(n, W, src, dist, iterations_ptr, stream)


def gemv(A, x, semiring="min", trans=False, out=None, accumulate=False, stream=None):
    """trans=False: y_i = (+)_j A[i,j] (.) x_j; trans=True: y_j = (+)_i x_i (.) A[i,j]."""
    torch = _torch()
    m, n = A.shape
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs `out`")
        out = torch.empty(n if trans else m, dtype=A.dtype, device=A.device)
    flags = _sr(semiring) | (GEMM_ACCUMULATE if accumulate else 0)
    check(btas_gemv(flags, _dtype_code(A), 1 if trans else 0, m, n, A.data_ptr(), _rowmajor(A, "A"), x.data_ptr(),
                    out.data_ptr(), _stream(stream)))
    return out


def sssp(W, src, stream=None, info=False):
    """Single-source shortest paths (Bellman-Ford by repeated min-plus
    vector-matrix products) from vertex `src` of the int32 matrix W."""
    torch = _torch()
    n = W.shape[0]
    d = torch.empty(n, dtype=torch.int32, device=W.device)
    it = ctypes.c_int(0)
    check(btas_sssp(n, W.data_ptr(), int(src), d.data_ptr(), ctypes.addressof(it), _stream(stream)))
    return (d, {"iterations": it.value}) if info else d


def btas_apsp_noalloc(n, W, D, stream) -> int:
    return lib().btas_apsp_noalloc(n, W, D, stream)


def btas_apsp_noalloc_status(stream, squarings_done_ptr) -> int:
    return lib().btas_apsp_noalloc_status(stream, squarings_done_ptr)


def btas_batch_create(out_ptr, flags) -> int:
    return lib().btas_batch_create(out_ptr, flags)


def btas_batch_add_apsp(b, n, W, D) -> int:
    return lib().btas_batch_add_apsp(b, n, W, D)


def btas_batch_add_gemm(b, semiring, dtype, m, n, k, A, lda, B, ldb, C, ldc) -> int:
    return lib().btas_batch_add_gemm(b, semiring, dtype, m, n, k, A, lda, B, ldb, C, ldc)


def btas_batch_launch(b, stream) -> int:
    return lib().btas_batch_launch(b, stream)


def btas_batch_wait(b, stream) -> int:
    return lib().btas_batch_wait(b, stream)


def btas_batch_destroy(b) -> int:
    return lib().btas_batch_destroy(b)


def btas_batch_workspace_bytes(b) -> int:
    return lib().btas_batch_workspace_bytes(b)


def btas_batch_tasks(b) -> int:
    return lib().btas_batch_tasks(b)


def btas_batch_profile(b, cycles_ptr, counts_ptr, slots) -> int:
    return lib().btas_batch_profile(b, cycles_ptr, counts_ptr, slots)


def btas_batch_tune(n_max, stream, ms_ptr, max_entries) -> int:
    return lib().btas_batch_tune(n_max, stream, ms_ptr, max_entries)


def btas_batch_tile(kind, n) -> int:
    return lib().btas_batch_tile(kind, n)


def btas_batch_tune_clear() -> None:
    lib().btas_batch_tune_clear()


def btas_batch_select_tiles(b, stream, mode_ptr, ms_ptr) -> int:
    return lib().btas_batch_select_tiles(b, stream, mode_ptr, ms_ptr)


BATCH_TILE_KINDS = ("apsp", "i32_product", "f32_product")


def batch_tune(n_max=1024, stream=None):
    """Tile autotuner of the batched launch (btas_batch_tune).  Returns
    {kind: [(bucket_lo, bucket_hi, tile, ms_128, ms_64), ...]}."""
    buckets = (n_max + 31) // 32
    ms = (ctypes.c_double * (2 * 3 * buckets))()
    check(btas_batch_tune(n_max, _stream(stream), ctypes.addressof(ms), 2 * 3 * buckets))
    out = {}
    for kind, name in enumerate(BATCH_TILE_KINDS):
        rows = []
        for b in range(buckets):
            lo, hi = 32 * b + 1, min(n_max, 32 * b + 32)
            rows.append((lo, hi, btas_batch_tile(kind, hi), round(ms[2 * (kind * buckets + b)], 4),
                         round(ms[2 * (kind * buckets + b) + 1], 4)))
        out[name] = rows
    return out


# ------------------------------------------------------- torch helpers
_torch_mod = None


def _torch():
    global _torch_mod
    if _torch_mod is None:
        import torch
        _torch_mod = torch
    return _torch_mod


def _stream(stream=None) -> int:
    """The cudaStream_t of `stream`, or of the current device's current stream
    (read without building a Stream object: this is on every call's path)."""
    if stream is not None:
        return int(stream.cuda_stream)
    torch = _torch()
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    if raw is not None:
        return int(raw(torch.cuda.current_device()))
    return int(torch.cuda.current_stream().cuda_stream)


def _sr(semiring) -> int:
    if semiring in (MINPLUS, "min", "minplus", "min-plus"):
        return MINPLUS
    if semiring in (MAXPLUS, "max", "maxplus", "max-plus"):
        return MAXPLUS
    raise ValueError(f"unknown semiring {semiring!r}")


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.float32:
        return F32
    if t.dtype in (torch.int16, getattr(torch, "uint16", torch.int16)):
        return U16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _rowmajor(t, name):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a 2-D row-major tensor (unit column stride)")
    return max(t.stride(0), 1) if t.shape[0] > 1 else max(t.shape[1], 1)


def gemm(A, B, semiring="min", out=None, accumulate=False, trans_b=False, stream=None, no_carrier=False,
         packed=False, checked=False):
    """Tropical product C = A (x) B (or C (+)= A (x) B with accumulate).

    A, B are CUDA tensors (int32, float32, or int16 holding values in
    [0, 0x7FFF] for the packed min-plus path).  With trans_b, B is given as
    B^T (n x k).  With packed=True (int32) the product runs on the exact
    packed 16-bit kernel when the operands' finite ranges allow it
    (BTAS_GEMM_PACKED; decided on the device, same bits either way).  With
    checked=True the operand domain is checked on the device
    (BTAS_GEMM_CHECKED): a violation leaves `out` unwritten and is reported
    by sync_status().  CPU
    tensors are copied to the current device and the result is copied back
    (host -> device -> kernel -> host, the flow of Fig. 1)."""
    torch = _torch()
    host = A.device.type == "cpu"
    if host:
        dev = torch.device("cuda", torch.cuda.current_device())
        Ad, Bd = A.to(dev, non_blocking=True), B.to(dev, non_blocking=True)
        od = out.to(dev, non_blocking=True) if (out is not None and accumulate) else None
        C = gemm(Ad, Bd, semiring, od, accumulate, trans_b, stream, no_carrier, packed, checked)
        if out is None:
            return C.cpu()
        out.copy_(C)
        return out
    m, k = A.shape
    n = B.shape[0] if trans_b else B.shape[1]
    if (B.shape[1] if trans_b else B.shape[0]) != k:
        raise ValueError("inner dimensions differ")
    if out is None:
        if accumulate:
            raise ValueError("accumulate needs `out`")
        out = torch.empty((m, n), dtype=A.dtype, device=A.device)
    flags = _sr(semiring) | (GEMM_ACCUMULATE if accumulate else 0) | (GEMM_TRANS_B if trans_b else 0)
    flags |= GEMM_NO_CARRIER if no_carrier else 0
    flags |= GEMM_PACKED if packed else 0
    flags |= GEMM_CHECKED if checked else 0
    check(btas_gemm(flags, _dtype_code(A), m, n, k, A.data_ptr(), _rowmajor(A, "A"), B.data_ptr(),
                    _rowmajor(B, "B"), out.data_ptr(), _rowmajor(out, "out"), _stream(stream)))
    return out


def btas_sync_status(stream, out_of_domain_ptr, calls_ptr) -> int:
    return lib().btas_sync_status(stream, out_of_domain_ptr, calls_ptr)


def sync_status(stream=None):
    """Device-side errors of asynchronous calls (btas_sync_status):
    synchronises the stream, clears the device's status words and returns
    (status, out_of_domain_entries, checked_calls_that_found_any)."""
    e, c = ctypes.c_int64(0), ctypes.c_int64(0)
    st = btas_sync_status(_stream(stream), ctypes.addressof(e), ctypes.addressof(c))
    return st, e.value, c.value


def apsp(W, out=None, flags=APSP_EARLY_EXIT, stream=None, info=False):
    """All-pairs shortest paths of the int32 adjacency matrix W by repeated
    min-plus squaring (Sec. III).  out may be W (in place).  With info=True
    returns (D, {"squarings": ..., "bound": ..., "path": ...})."""
    torch = _torch()
    n = W.shape[0]
    if W.shape != (n, n) or not W.is_contiguous() or W.dtype != torch.int32:
        raise ValueError("W must be a contiguous n x n int32 tensor")
    if out is None:
        out = torch.empty_like(W)
    sq, bd, pt = ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_int(0)
    if info:
        check(btas_apsp_ex(n, W.data_ptr(), out.data_ptr(), flags, ctypes.addressof(sq), ctypes.addressof(bd),
                           ctypes.addressof(pt), _stream(stream)))
        names = [nm for bit, nm in ((1, "int32"), (2, "fp32-carrier"), (4, "u16x2"), (8, "sparse")) if pt.value & bit]
        return out, {"squarings": sq.value, "bound": bd.value, "path": "+".join(names)}
    if flags == APSP_EARLY_EXIT:
        check(btas_apsp(n, W.data_ptr(), out.data_ptr(), _stream(stream)))
    else:
        check(btas_apsp_ex(n, W.data_ptr(), out.data_ptr(), flags, None, None, None, _stream(stream)))
    return out


def apsp_u16(W, max_w, out=None, early_exit=True, stream=None):
    """APSP on 16-bit storage (INF = 0x7FFF) through the packed path; requires
    (n-1) * max_w < 0x7FFF."""
    torch = _torch()
    n = W.shape[0]
    if out is None:
        out = torch.empty_like(W)
    check(btas_apsp_u16(n, W.data_ptr(), out.data_ptr(), int(max_w), APSP_EARLY_EXIT if early_exit else 0,
                        _stream(stream)))
    return out


def dot(x, y, semiring="min", incx=1, incy=1, n=None, out=None, stream=None):
    torch = _torch()
    if n is None:
        n = (x.numel() + incx - 1) // incx
    if out is None:
        out = torch.empty((), dtype=x.dtype, device=x.device)
    check(btas_dot(_sr(semiring), _dtype_code(x), n, x.data_ptr(), incx, y.data_ptr(), incy, out.data_ptr(),
                   _stream(stream)))
    return out


def axpy(alpha, x, y, semiring="min", incx=1, incy=1, n=None, stream=None):
    """y <- y (+) (alpha (.) x), in place on y."""
    if n is None:
        n = (x.numel() + incx - 1) // incx
    code = _dtype_code(x)
    a = ctypes.c_int32(int(alpha)) if code == I32 else ctypes.c_float(float(alpha))
    check(btas_axpy(_sr(semiring), code, n, ctypes.addressof(a), x.data_ptr(), incx, y.data_ptr(), incy,
                    _stream(stream)))
    return y


def add(x, y, semiring="min", out=None, stream=None):
    torch = _torch()
    out = torch.empty_like(x) if out is None else out
    check(btas_add(_sr(semiring), _dtype_code(x), x.numel(), x.data_ptr(), y.data_ptr(), out.data_ptr(),
                   _stream(stream)))
    return out


def mul(x, y, semiring="min", out=None, stream=None):
    torch = _torch()
    out = torch.empty_like(x) if out is None else out
    check(btas_mul(_sr(semiring), _dtype_code(x), x.numel(), x.data_ptr(), y.data_ptr(), out.data_ptr(),
                   _stream(stream)))
    return out


BATCH_NO_GRAPH = 0x1


class Batch:
    """Many APSP solves and tropical products in one persistent launch
    (btas_batch_*).  Keep the tensors alive until `wait()` returns."""

    def __init__(self, graph: bool = True, profile: bool = False):
        h = ctypes.c_void_p()
        flags = (0 if graph else BATCH_NO_GRAPH) | (BATCH_PROFILE if profile else 0)
        check(btas_batch_create(ctypes.addressof(h), flags))
        self.handle = h.value
        self._keep = []

    def add_apsp(self, W, D):
        torch = _torch()
        n = W.shape[0]
        if W.dtype != torch.int32 or W.shape != (n, n) or not W.is_contiguous() or not D.is_contiguous():
            raise ValueError("W, D must be contiguous n x n int32 tensors")
        check(btas_batch_add_apsp(self.handle, n, W.data_ptr(), D.data_ptr()))
        self._keep += [W, D]
        return D

    def add_gemm(self, A, B, C, semiring="min", trans_b=False):
        m, k = A.shape
        n = B.shape[0] if trans_b else B.shape[1]
        flags = _sr(semiring) | (GEMM_TRANS_B if trans_b else 0)
        check(btas_batch_add_gemm(self.handle, flags, _dtype_code(A), m, n, k, A.data_ptr(), _rowmajor(A, "A"),
                                  B.data_ptr(), _rowmajor(B, "B"), C.data_ptr(), _rowmajor(C, "C")))
        self._keep += [A, B, C]
        return C

    def launch(self, stream=None):
        check(btas_batch_launch(self.handle, _stream(stream)))

    def wait(self, stream=None):
        check(btas_batch_wait(self.handle, _stream(stream)))

    @property
    def tasks(self) -> int:
        return btas_batch_tasks(self.handle)

    def select_tiles(self, stream=None):
        """btas_batch_select_tiles: times the batch with the tuned table's
        tiles, all 128 x 128 and all 64 x 64, keeps the fastest; returns
        (mode name, {mode: ms})."""
        mode = ctypes.c_int(0)
        ms = (ctypes.c_double * 3)()
        check(btas_batch_select_tiles(self.handle, _stream(stream), ctypes.addressof(mode), ctypes.addressof(ms)))
        names = ("table", "all_128x128", "all_64x64")
        return names[mode.value], {nm: round(ms[i], 3) for i, nm in enumerate(names)}

    def profile(self) -> dict:
        """Per-task-kind SM cycles and task counts, summed over every launch
        (batch created with profile=True); synchronises the device."""
        cyc = (ctypes.c_uint64 * BATCH_PROFILE_SLOTS)()
        cnt = (ctypes.c_uint64 * BATCH_PROFILE_SLOTS)()
        check(lib().btas_batch_profile(self.handle, ctypes.addressof(cyc), ctypes.addressof(cnt),
                                       BATCH_PROFILE_SLOTS))
        return {name: {"cycles": int(cyc[i]), "tasks": int(cnt[i])} for i, name in enumerate(BATCH_SLOT_NAMES)}

    @property
    def workspace_bytes(self) -> int:
        return btas_batch_workspace_bytes(self.handle)

    def close(self):
        if self.handle:
            btas_batch_destroy(self.handle)
            self.handle = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (btas_server_*).  Submit requests
    with host tensors (pinned for asynchronous copies); keep them alive until
    the request is done."""

    def __init__(self, hbm_budget_bytes: int):
        h = ctypes.c_void_p()
        check(lib().btas_server_create(ctypes.addressof(h), int(hbm_budget_bytes), 0))
        self.handle = h.value
        self._keep = {}

    def submit_apsp(self, W, D) -> int:
        n = W.shape[0]
        if W.device.type != "cpu" or D.device.type != "cpu" or not W.is_contiguous() or not D.is_contiguous():
            raise ValueError("server requests take contiguous host tensors")
        t = ctypes.c_int64()
        check(lib().btas_server_submit_apsp(self.handle, n, W.data_ptr(), D.data_ptr(), ctypes.addressof(t)))
        self._keep[t.value] = (W, D)
        return t.value

    def submit_gemm(self, A, B, C, semiring="min") -> int:
        m, k = A.shape
        n = B.shape[1]
        for x in (A, B, C):
            if x.device.type != "cpu" or not x.is_contiguous():
                raise ValueError("server requests take contiguous host tensors")
        t = ctypes.c_int64()
        check(lib().btas_server_submit_gemm(self.handle, _sr(semiring), _dtype_code(A), m, n, k, A.data_ptr(),
                                            B.data_ptr(), C.data_ptr(), ctypes.addressof(t)))
        self._keep[t.value] = (A, B, C)
        return t.value

    def poll(self, ticket: int):
        st = ctypes.c_int()
        ts, ta, td = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().btas_server_poll(self.handle, ticket, ctypes.addressof(st), ctypes.addressof(ts),
                                     ctypes.addressof(ta), ctypes.addressof(td)))
        return {"state": st.value, "t_submit": ts.value, "t_admit": ta.value, "t_done": td.value}

    def wait_all(self, timeout_s: float = 600.0):
        check(lib().btas_server_wait_all(self.handle, float(timeout_s)))

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        check(lib().btas_server_stats(self.handle, *[ctypes.addressof(x) for x in v]))
        return {"steps": v[0].value, "units": v[1].value, "completed": v[2].value, "bytes_in_use": v[3].value}

    def close(self):
        if self.handle:
            lib().btas_server_destroy(self.handle)
            self.handle = None
            self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ autotuner
def btas_tune_gemm(semiring, dtype, m, n, k, out_ptr, stream) -> int:
    return lib().btas_tune_gemm(semiring, dtype, m, n, k, out_ptr, stream)


def btas_tune_lookup(semiring, dtype, m, n, k, out_ptr) -> int:
    return lib().btas_tune_lookup(semiring, dtype, m, n, k, out_ptr)


def btas_tune_save(path) -> int:
    return lib().btas_tune_save(os.fsencode(path))


def btas_tune_load(path, loaded_ptr) -> int:
    return lib().btas_tune_load(os.fsencode(path), loaded_ptr)


def btas_tune_clear() -> None:
    lib().btas_tune_clear()


def btas_tune_entries() -> int:
    return lib().btas_tune_entries()


def tune_gemm(semiring, dtype, m, n, k, stream=None) -> dict:
    """Time every compiled kernel for (semiring, dtype) at m x n x k, keep the
    fastest in the tuning table and return it as a dict (btas_tune_result)."""
    r = TuneResult()
    check(btas_tune_gemm(_sr(semiring), dtype, m, n, k, ctypes.addressof(r), _stream(stream)))
    return r.as_dict()


def tune_lookup(semiring, dtype, m, n, k):
    """The table's entry for this problem's size buckets on the current
    device, or None."""
    r = TuneResult()
    return r.as_dict() if btas_tune_lookup(_sr(semiring), dtype, m, n, k, ctypes.addressof(r)) else None


def tune_save(path) -> None:
    check(btas_tune_save(path))


def tune_load(path) -> int:
    c = ctypes.c_int()
    check(btas_tune_load(path, ctypes.addressof(c)))
    return c.value


def tune_clear() -> None:
    btas_tune_clear()


def tune_entries() -> int:
    return btas_tune_entries()
