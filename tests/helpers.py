"""Shared test helpers: error metric, tolerances, GPU round trips through the C ABI."""
from __future__ import annotations

import math
import os

import numpy as np

FP32_TOL_PER_LOG2N = 2e-7   # plain FP32 path: rel-L2 <= 2e-7 * log2(N)
TC_TOL_PER_LOG2N = 1e-6     # split-precision tensor-core path: <= 1e-6 * log2(N)


def tol_fp32(n: int) -> float:
    return FP32_TOL_PER_LOG2N * max(1.0, math.log2(n))


def row_rel_l2(y, ref) -> np.ndarray:
    """Per-row relative L2 error ||y - ref|| / ||ref|| (absolute if ||ref|| = 0), in FP64."""
    y = np.asarray(y, dtype=np.complex128).reshape(-1, np.asarray(ref).shape[-1])
    ref = np.asarray(ref, dtype=np.complex128).reshape(y.shape)
    num = np.linalg.norm(y - ref, axis=1)
    den = np.linalg.norm(ref, axis=1)
    return np.where(den > 0, num / np.where(den > 0, den, 1.0), num)


def ncpu() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def to_device(x: np.ndarray):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex64).view(np.float32).reshape(-1))
    return t.to("cuda")


def from_device(t, shape) -> np.ndarray:
    return t.cpu().numpy().view(np.complex64).reshape(shape)


def gpu_fft(x: np.ndarray, direction: int = -1, variant=None, inplace: bool = False) -> np.ndarray:
    """Run the library on a (batch, n) complex64 array and return the result."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, n = x.shape
    d_in = to_device(x)
    d_out = d_in if inplace else torch.empty_like(d_in)
    with gbfft.Plan(n, batch, direction, variant=variant) as p:
        p.execute(d_in, d_out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
    return from_device(d_out, (batch, n))
