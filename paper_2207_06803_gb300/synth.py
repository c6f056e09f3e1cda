"""Seeded synthetic inputs for the batched complex DFT.

This module is the one piece shared by the GPU library's tests/benchmarks and
the CPU oracle.  It holds no part of the transform's arithmetic: it only turns
(seed, element index) into complex64 sample values, so any row of any batch can
be regenerated on the host from its indices alone, without copying the device
buffer back.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used as a counter-based generator: the c-th
word of a stream is the finaliser applied to ``seed + (c + 1) * 0x9E3779B97F4A7C15``
(mod 2^64), i.e. the (c+1)-th output of SplitMix64 started from ``seed``.

Distributions (the paper's inputs are "random input vectors"; its workloads are
small one-dimensional transforms):

* ``uniform``: complex element ``e`` of the flat buffer has real part U(2e) and
  imaginary part U(2e+1), ``U(c) = (word(c) >> 40) * 2^-23 - 1``: a 24-bit
  lattice in [-1, 1), every value exactly representable in float32.  Because
  the counter is the flat element index, the flat buffer is the same for every
  row length, and row ``i`` of a batch of rows of length ``n`` is elements
  ``[i*n, (i+1)*n)``.
* ``gaussian_scaled``: Box-Muller normals (FP64, rounded to float32) from the
  word stream of ``seed ^ GAUSS_SALT``, each row multiplied by ``10**s`` with
  ``s`` uniform in [-3, 3) drawn from the word stream of ``seed ^ SCALE_SALT``
  at counter = row index.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20220714
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
GAUSS_SALT = 0x6A09E667F3BCC908
SCALE_SALT = 0xBB67AE8584CAA73B
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22  # counters per vectorised chunk (bounds host temporaries)


def words(seed: int, start: int, count: int) -> np.ndarray:
    """SplitMix64 words for counters ``start .. start+count-1`` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, count, _CHUNK):
            hi = min(count, lo + _CHUNK)
            z = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            z *= GOLDEN
            z += s
            z ^= z >> np.uint64(30)
            z *= _M1
            z ^= z >> np.uint64(27)
            z *= _M2
            z ^= z >> np.uint64(31)
            out[lo:hi] = z
    return out


def _unit_lattice(w: np.ndarray) -> np.ndarray:
    """24-bit uniform in [-1, 1): (w >> 40) * 2^-23 - 1, exact in float32."""
    return ((w >> np.uint64(40)).astype(np.float64) * (2.0 ** -23) - 1.0).astype(np.float32)


def uniform_flat(seed: int, start: int, count: int) -> np.ndarray:
    """Complex64 elements ``start .. start+count-1`` of the uniform flat stream."""
    w = words(seed, 2 * start, 2 * count)
    out = np.empty(count, dtype=np.complex64)
    f = out.view(np.float32)
    f[:] = _unit_lattice(w)
    return out


def uniform_rows(seed: int, n: int, rows) -> np.ndarray:
    """Rows (given by index) of a contiguous batch of length-``n`` rows."""
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    out = np.empty((rows.size, n), dtype=np.complex64)
    for i, r in enumerate(rows):
        out[i] = uniform_flat(seed, int(r) * n, n)
    return out


def uniform_batch(seed: int, n: int, batch: int) -> np.ndarray:
    """A full ``(batch, n)`` complex64 batch of the uniform stream."""
    return uniform_flat(seed, 0, n * batch).reshape(batch, n)


def _row_scales(seed: int, rows: np.ndarray) -> np.ndarray:
    s = np.uint64((seed ^ SCALE_SALT) & 0xFFFFFFFFFFFFFFFF)
    out = np.empty(rows.size, dtype=np.float64)
    for i, r in enumerate(rows):
        w = words(int(s), int(r), 1)
        u = (w >> np.uint64(40)).astype(np.float64) * (2.0 ** -23) - 1.0  # [-1, 1)
        out[i] = 10.0 ** (3.0 * u[0])
    return out


def gaussian_scaled_rows(seed: int, n: int, rows) -> np.ndarray:
    """Rows of a batch whose samples are standard complex normals (Box-Muller)
    times a per-row scale 10^U(-3,3)."""
    rows = np.atleast_1d(np.asarray(rows, dtype=np.int64))
    gs = (seed ^ GAUSS_SALT) & 0xFFFFFFFFFFFFFFFF
    scales = _row_scales(seed, rows)
    out = np.empty((rows.size, n), dtype=np.complex64)
    for i, r in enumerate(rows):
        w = words(gs, 2 * int(r) * n, 2 * n)
        u1 = ((w[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
        u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)          # [0, 1)
        rad = np.sqrt(-2.0 * np.log(u1)) * scales[i]
        ang = 2.0 * np.pi * u2
        out[i].real = (rad * np.cos(ang)).astype(np.float32)
        out[i].imag = (rad * np.sin(ang)).astype(np.float32)
    return out


def gaussian_scaled_batch(seed: int, n: int, batch: int) -> np.ndarray:
    """A full ``(batch, n)`` complex64 batch of scaled Gaussian rows."""
    gs = (seed ^ GAUSS_SALT) & 0xFFFFFFFFFFFFFFFF
    w = words(gs, 0, 2 * n * batch)
    u1 = ((w[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (w[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    del w
    rad = np.sqrt(-2.0 * np.log(u1)).reshape(batch, n)
    rad *= _row_scales_vec(seed, batch)[:, None]
    ang = (2.0 * np.pi) * u2.reshape(batch, n)
    out = np.empty((batch, n), dtype=np.complex64)
    out.real = (rad * np.cos(ang)).astype(np.float32)
    out.imag = (rad * np.sin(ang)).astype(np.float32)
    return out


def _row_scales_vec(seed: int, batch: int) -> np.ndarray:
    s = (seed ^ SCALE_SALT) & 0xFFFFFFFFFFFFFFFF
    w = words(s, 0, batch)
    u = (w >> np.uint64(40)).astype(np.float64) * (2.0 ** -23) - 1.0
    return 10.0 ** (3.0 * u)


def sample_rows(seed: int, batch: int, count: int) -> np.ndarray:
    """``count`` distinct row indices in [0, batch), chosen by a seeded shuffle."""
    count = min(count, batch)
    rng = np.random.Generator(np.random.Philox(key=seed & 0xFFFFFFFFFFFFFFFF))
    return np.sort(rng.choice(batch, size=count, replace=False)).astype(np.int64)


# ---------------------------------------------------------------------------
# Ragged batches: transform lengths of the form 2^k, 3*2^k, 5*2^k, 7*2^k.
# ---------------------------------------------------------------------------

def size_family(lo: int, hi: int) -> list[int]:
    """Sorted sizes {2^k, 3*2^k, 5*2^k, 7*2^k} within [lo, hi]."""
    out = set()
    for base in (1, 3, 5, 7):
        v = base
        while v <= hi:
            if v >= lo:
                out.add(v)
            v *= 2
    return sorted(out)


def ragged_sizes(seed: int, count: int, lo: int = 8, hi: int = 8192) -> np.ndarray:
    """``count`` lengths drawn uniformly from :func:`size_family` (lo, hi).  The
    family has four sizes per octave, so the draw is close to log-uniform."""
    fam = np.asarray(size_family(lo, hi), dtype=np.int64)
    rng = np.random.Generator(np.random.Philox(key=(seed ^ 0xA5A5A5A5) & 0xFFFFFFFFFFFFFFFF))
    return fam[rng.integers(0, fam.size, size=count)]


def ragged_offsets(sizes: np.ndarray) -> np.ndarray:
    """Exclusive prefix sum: transform i starts at complex element offsets[i]."""
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.size, dtype=np.int64)
    if sizes.size > 1:
        np.cumsum(sizes[:-1], out=off[1:])
    return off
