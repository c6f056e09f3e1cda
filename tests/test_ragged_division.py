"""The ragged kernel divides by run-time invariants (n/R, L, n) with a
multiply-high: m = ceil(2^31 / d), floor(x / d) = (2x * m) >> 32 (Granlund and
Montgomery, 1994).  Exhaustive on the host for every divisor 1..8192 and every
dividend below 8192 (the tile bound), in the kernel's 32-bit arithmetic."""
import numpy as np


def test_multiply_high_division_is_exact_below_the_tile_bound():
    x = np.arange(8192, dtype=np.uint64)
    for d in range(1, 8193):
        m = ((1 << 31) + d - 1) // d
        assert m < (1 << 32)
        two_x = (x << np.uint64(1)) & np.uint64(0xFFFFFFFF)  # (unsigned)x << 1
        q = (two_x * np.uint64(m)) >> np.uint64(32)          # __umulhi
        assert np.array_equal(q, x // np.uint64(d)), d
