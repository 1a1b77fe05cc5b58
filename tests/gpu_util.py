"""Helpers shared by the GPU parity tests (device placement, bit views)."""
import numpy as np

import gen

INF = 0x3FFFFFFF
NINF = -0x3FFFFFFF


def torch_mod():
    import torch
    return torch


def dev(a: np.ndarray):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy()


def bits(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


def int_matrix(seed, shape, sr, lo=-1000, hi=1000, p_inf=0.1):
    v = gen.uniform_int(seed, 1, shape, lo, hi)
    if p_inf:
        u = gen.uniform_unit_f64(seed, 2, np.arange(v.size, dtype=np.uint64)).reshape(shape)
        v = np.where(u < p_inf, INF if sr == 0 else NINF, v).astype(np.int32)
    return v


def f32_matrix(seed, shape, sr, p_inf=0.1):
    v = gen.uniform_f32(seed, 3, shape) * np.float32(4.0) - np.float32(1.0)
    if p_inf:
        u = gen.uniform_unit_f64(seed, 4, np.arange(v.size, dtype=np.uint64)).reshape(shape)
        v = np.where(u < p_inf, np.float32(np.inf if sr == 0 else -np.inf), v).astype(np.float32)
    return v
