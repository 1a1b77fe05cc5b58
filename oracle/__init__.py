"""CPU oracle for the tropical-algebra hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline leg
import this package.  The library (`paper_1701_04733_gb300`) never does, and
the two share no code: this package compiles `btas_oracle.c` with gcc and
calls it through ctypes on numpy arrays.

What each function computes, and the passage it follows:
  tgemm(sr, A, B)             C = A (x) B, the (+)-sum over k of A[i,k] (.) B[k,j]
                              (Eq. 1-4; the matrix-product listing of Sec. IV)
  tgemm_u16(A, B)             16-bit min-plus product saturating at INF16
  apsp_squarings(n)           S = ceil(log2(n-1)) (Sec. III)
  apsp_squaring(W)            D = W squared S times (Sec. III)
  floyd_warshall(W)           Algorithm 2 with an INF sentinel
  apsp_paths(W)               squaring with next-hop matrix (smallest minimising k)
  dijkstra_rows(W, srcs)      textbook single-source shortest paths
  gemv(sr, A, x, trans)       tropical matrix-vector product (level 2)
  sssp(W, src)                Bellman-Ford as repeated min-plus vector-matrix products
  bruteforce_apsp(W)          minimum over all simple paths (n <= 8)
  dot / axpy / add / mul      tropical vector operations (abstract, Sec. III)

Every function is pinned by tests in tests/test_oracle_*.py against closed
forms, invariants, brute force and independent textbook algorithms.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btas_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libbtas_oracle.so")

MINPLUS = 0
MAXPLUS = 1
INF_I32 = 0x3FFFFFFF
NINF_I32 = -0x3FFFFFFF
INF_U16 = 0x7FFF

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile btas_oracle.c into a shared library (gcc, OpenMP, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        sig = {
            "oracle_set_threads": (None, [i32]),
            "oracle_get_threads": (i32, []),
            "oracle_tgemm_i32": (None, [i32, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64]),
            "oracle_tgemm_f32": (None, [i32, i32, i64, i64, i64, vp, i64, vp, i64, vp, i64]),
            "oracle_tgemm_u16": (None, [i32, i64, i64, i64, vp, i64, vp, i64, vp, i64]),
            "oracle_apsp_squarings": (i32, [i64]),
            "oracle_apsp_squaring_i32": (None, [i64, vp, vp, i32]),
            "oracle_apsp_squaring_u16": (None, [i64, vp, vp, i32]),
            "oracle_fw_i32": (None, [i64, vp]),
            "oracle_apsp_paths_i32": (None, [i64, vp, vp, vp, i32]),
            "oracle_apsp_paths_f32": (None, [i64, vp, vp, vp, i32]),
            "oracle_dijkstra_rows_i32": (None, [i64, vp, i64, vp, vp]),
            "oracle_bruteforce_apsp_i32": (i32, [i64, vp, vp]),
            "oracle_gemv_i32": (None, [i32, i32, i32, i64, i64, vp, i64, vp, vp]),
            "oracle_gemv_f32": (None, [i32, i32, i32, i64, i64, vp, i64, vp, vp]),
            "oracle_sssp_i32": (i32, [i64, vp, i64, vp]),
            "oracle_dot_i32": (ctypes.c_int32, [i32, i64, vp, i64, vp, i64]),
            "oracle_dot_f32": (ctypes.c_float, [i32, i64, vp, i64, vp, i64]),
            "oracle_axpy_i32": (None, [i32, i64, ctypes.c_int32, vp, i64, vp, i64]),
            "oracle_axpy_f32": (None, [i32, i64, ctypes.c_float, vp, i64, vp, i64]),
            "oracle_add_i32": (None, [i32, i64, vp, vp, vp]),
            "oracle_mul_i32": (None, [i32, i64, vp, vp, vp]),
            "oracle_add_f32": (None, [i32, i64, vp, vp, vp]),
            "oracle_mul_f32": (None, [i32, i64, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def set_threads(t: int) -> None:
    """Threads used by the row-parallel loops (default 1)."""
    _load().oracle_set_threads(int(t))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def tgemm(sr: int, A: np.ndarray, B: np.ndarray, C: np.ndarray | None = None) -> np.ndarray:
    """Tropical product A (x) B (int32 or float32).  With C given, returns C (+) A (x) B."""
    A = np.asarray(A)
    dt = np.int32 if A.dtype.kind in "iu" else np.float32
    A = _c(A, dt)
    B = _c(B, dt)
    m, k = A.shape
    k2, n = B.shape
    assert k == k2
    acc = C is not None
    out = _c(C, dt).copy() if acc else np.empty((m, n), dtype=dt)
    f = _load().oracle_tgemm_i32 if dt == np.int32 else _load().oracle_tgemm_f32
    f(sr, int(acc), m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(out), max(n, 1))
    return out


def tgemm_u16(A: np.ndarray, B: np.ndarray, C: np.ndarray | None = None) -> np.ndarray:
    """16-bit min-plus product saturating at INF16 = 0x7FFF."""
    A = _c(A, np.uint16)
    B = _c(B, np.uint16)
    m, k = A.shape
    _, n = B.shape
    acc = C is not None
    out = _c(C, np.uint16).copy() if acc else np.empty((m, n), dtype=np.uint16)
    _load().oracle_tgemm_u16(int(acc), m, n, k, _p(A), max(k, 1), _p(B), max(n, 1),
                             _p(out), max(n, 1))
    return out


def apsp_squarings(n: int) -> int:
    return int(_load().oracle_apsp_squarings(int(n)))


def apsp_squaring(W: np.ndarray, squarings: int | None = None) -> np.ndarray:
    """APSP by repeated min-plus squaring of W (int32 or uint16)."""
    n = W.shape[0]
    s = apsp_squarings(n) if squarings is None else int(squarings)
    if W.dtype == np.uint16:
        W = _c(W, np.uint16)
        D = np.empty_like(W)
        _load().oracle_apsp_squaring_u16(n, _p(W), _p(D), s)
        return D
    W = _c(W, np.int32)
    D = np.empty_like(W)
    _load().oracle_apsp_squaring_i32(n, _p(W), _p(D), s)
    return D


def apsp_paths(W: np.ndarray, squarings: int | None = None):
    """APSP by squaring with next-hop tracking (smallest minimising k), int32
    or float32 weights.  Returns (D, Next)."""
    W = np.asarray(W)
    dt = np.float32 if W.dtype.kind == "f" else np.int32
    W = _c(W, dt)
    n = W.shape[0]
    s = apsp_squarings(n) if squarings is None else int(squarings)
    D = np.empty_like(W)
    Nx = np.empty(W.shape, dtype=np.int32)
    fn = _load().oracle_apsp_paths_f32 if dt == np.float32 else _load().oracle_apsp_paths_i32
    fn(n, _p(W), _p(D), _p(Nx), s)
    return D, Nx


def floyd_warshall(W: np.ndarray) -> np.ndarray:
    D = _c(W, np.int32).copy()
    _load().oracle_fw_i32(D.shape[0], _p(D))
    return D


def dijkstra_rows(W: np.ndarray, srcs) -> np.ndarray:
    W = _c(W, np.int32)
    srcs = np.ascontiguousarray(srcs, dtype=np.int64)
    n = W.shape[0]
    rows = np.empty((len(srcs), n), dtype=np.int32)
    _load().oracle_dijkstra_rows_i32(n, _p(W), len(srcs), _p(srcs), _p(rows))
    return rows


def bruteforce_apsp(W: np.ndarray) -> np.ndarray:
    W = _c(W, np.int32)
    D = np.empty_like(W)
    rc = _load().oracle_bruteforce_apsp_i32(W.shape[0], _p(W), _p(D))
    if rc != 0:
        raise ValueError("brute force is limited to n <= 8")
    return D


def gemv(sr: int, A: np.ndarray, x: np.ndarray, trans: bool = False, y: np.ndarray | None = None):
    """trans=False: y_i = (+)_j A[i,j] (.) x_j; trans=True: y_j = (+)_i x_i (.) A[i,j]."""
    dt = np.int32 if np.asarray(A).dtype.kind in "iu" else np.float32
    A = _c(A, dt)
    x = _c(x, dt)
    m, n = A.shape
    acc = y is not None
    out = _c(y, dt).copy() if acc else np.empty(n if trans else m, dtype=dt)
    f = _load().oracle_gemv_i32 if dt == np.int32 else _load().oracle_gemv_f32
    f(sr, int(trans), int(acc), m, n, _p(A), max(n, 1), _p(x), _p(out))
    return out


def sssp(W: np.ndarray, src: int):
    """Bellman-Ford by repeated min-plus vector-matrix products: (dist, changed steps)."""
    W = _c(W, np.int32)
    n = W.shape[0]
    d = np.empty(n, dtype=np.int32)
    steps = _load().oracle_sssp_i32(n, _p(W), int(src), _p(d))
    return d, int(steps)


def dot(sr: int, x: np.ndarray, y: np.ndarray, incx: int = 1, incy: int = 1, n: int | None = None):
    dt = np.int32 if np.asarray(x).dtype.kind in "iu" else np.float32
    x = _c(x, dt)
    y = _c(y, dt)
    if n is None:
        n = len(x) // incx if incx else 0
    f = _load().oracle_dot_i32 if dt == np.int32 else _load().oracle_dot_f32
    return dt(f(sr, n, _p(x), incx, _p(y), incy))


def axpy(sr: int, alpha, x: np.ndarray, y: np.ndarray, incx: int = 1, incy: int = 1,
         n: int | None = None) -> np.ndarray:
    dt = np.int32 if np.asarray(x).dtype.kind in "iu" else np.float32
    x = _c(x, dt)
    out = _c(y, dt).copy()
    if n is None:
        n = len(x) // incx
    if dt == np.int32:
        _load().oracle_axpy_i32(sr, n, int(alpha), _p(x), incx, _p(out), incy)
    else:
        _load().oracle_axpy_f32(sr, n, float(alpha), _p(x), incx, _p(out), incy)
    return out


def add(sr: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    dt = np.int32 if np.asarray(x).dtype.kind in "iu" else np.float32
    x, y = _c(x, dt), _c(y, dt)
    z = np.empty_like(x)
    f = _load().oracle_add_i32 if dt == np.int32 else _load().oracle_add_f32
    f(sr, len(x), _p(x), _p(y), _p(z))
    return z


def mul(sr: int, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    dt = np.int32 if np.asarray(x).dtype.kind in "iu" else np.float32
    x, y = _c(x, dt), _c(y, dt)
    z = np.empty_like(x)
    f = _load().oracle_mul_i32 if dt == np.int32 else _load().oracle_mul_f32
    f(sr, len(x), _p(x), _p(y), _p(z))
    return z
