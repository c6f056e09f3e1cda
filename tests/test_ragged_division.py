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


def test_the_library_multipliers_are_the_ones_checked(tmp_path):
    """The multipliers the ragged plans upload come from ragged_magic in
    ragged.cuh: compile a host program against that header, print its value for
    every divisor 1..8192, and check each against ceil(2^31 / d), the value the
    exhaustive check above proves exact."""
    import os
    import shutil
    import subprocess

    import pytest
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is needed to compile against the kernel header")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "magic.cu"
    src.write_text('#include <cstdio>\n#include "ragged.cuh"\n'
                   'int main() { for (int d = 1; d <= 8192; ++d) std::printf("%u\\n", gbfft::ragged_magic(d)); }\n')
    exe = tmp_path / "magic"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(root, "include"), "-I", os.path.join(root, "paper_2207_06803_gb300", "csrc"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == [((1 << 31) + d - 1) // d for d in range(1, 8193)]
