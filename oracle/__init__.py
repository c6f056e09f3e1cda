"""CPU FP64 oracle for the batched one-dimensional complex DFT.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  It
shares no code with the GPU library (``paper_2207_06803_gb300``) and neither
imports the other; the only thing both sides consume is the seeded input
generator, which holds none of the transform's arithmetic.

The arithmetic lives in ``oracle.c`` (plain C, FP64):

* :func:`dft_naive`  -- the DFT definition of Sec. II as a dense mat-vec,
  ``y[m] = sum_k omega_N^(m*k) x[k]``, ``omega_N = exp(-2*pi*i/N)``.
* :func:`fft_radix2` -- textbook recursive radix-2 decimation in time.
* :func:`fft_eq2`    -- the recursion of Eq. 2,
  ``DFT_N = (DFT_K (x) I_M) D^N_M (I_K (x) DFT_M) Pi^N_K``.

:func:`dft_nd` composes them: the multi-dimensional DFT of row-major arrays,
``DFT_{d0} (x) ... (x) DFT_{d(r-1)}`` (Table I's Kronecker product applied to
whole transforms), one axis at a time.

``sign`` is the exponent sign: -1 forward, +1 unnormalised inverse, so that
``inverse(forward(x)) == N * x``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FORWARD = -1
INVERSE = +1

_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-Wextra",
             "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                    ctypes.c_int, ctypes.c_int]
        for name in ("oracle_dft_naive", "oracle_fft_radix2", "oracle_fft_eq2"):
            fn = getattr(lib, name)
            fn.argtypes = argtypes
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _run(name: str, x, sign: int, nthreads: int) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x), dtype=np.complex128)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[None, :]
    if x.ndim != 2:
        raise ValueError("expected a 1-D row or a 2-D (batch, n) array")
    batch, n = x.shape
    y = np.empty_like(x)
    rc = getattr(_load(), name)(x.ctypes.data, y.ctypes.data, n, batch, int(sign), int(nthreads))
    if rc != 0:
        raise ValueError(f"{name} failed with code {rc} (n={n}, batch={batch}, sign={sign})")
    return y[0] if squeeze else y


def dft_naive(x, sign: int = FORWARD, nthreads: int = 1) -> np.ndarray:
    """Direct O(N^2) DFT of each row (Sec. II definition), FP64."""
    return _run("oracle_dft_naive", x, sign, nthreads)


def fft_radix2(x, sign: int = FORWARD, nthreads: int = 1) -> np.ndarray:
    """Recursive radix-2 DIT FFT of each row; N must be a power of two."""
    return _run("oracle_fft_radix2", x, sign, nthreads)


def fft_eq2(x, sign: int = FORWARD, nthreads: int = 1) -> np.ndarray:
    """Recursive general-radix FFT following Eq. 2 (any N >= 1), FP64."""
    return _run("oracle_fft_eq2", x, sign, nthreads)


def dft(x, sign: int = FORWARD, nthreads: int = 1) -> np.ndarray:
    """The oracle's reference transform for checking a row: the direct DFT for
    N <= 1024 (cheap enough), else the Eq. 2 recursion (pinned to the direct
    DFT by the oracle's own tests)."""
    n = np.asarray(x).shape[-1]
    if n <= 1024:
        return dft_naive(x, sign, nthreads)
    return fft_eq2(x, sign, nthreads)


def dft_nd(x, sign: int = FORWARD, nthreads: int = 1) -> np.ndarray:
    """Multi-dimensional DFT of each item of a batch: x has shape
    (batch, d0, ..., d(r-1)), row-major.  The Kronecker product
    DFT_{d0} (x) ... (x) DFT_{d(r-1)} (Table I's operator on whole transforms)
    factors as (DFT_{d0} (x) I) (I (x) DFT_{d1} (x) I) ... , so the result is
    the 1-D transform of Sec. II along every axis in turn; each 1-D step is
    :func:`dft`.  The order of the axes does not matter (the factors commute)."""
    y = np.asarray(x, np.complex128)
    if y.ndim < 2:
        raise ValueError("expected (batch, d0, ..., d(r-1))")
    for ax in range(1, y.ndim):
        moved = np.moveaxis(y, ax, -1)
        shape = moved.shape
        out = dft(np.ascontiguousarray(moved).reshape(-1, shape[-1]), sign, nthreads).reshape(shape)
        y = np.moveaxis(out, -1, ax)
    return np.ascontiguousarray(y)
