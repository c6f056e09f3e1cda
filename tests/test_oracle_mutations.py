"""Planted mistakes: the oracle's pins must catch plausible slips.

Each case copies ``oracle/oracle.c`` to a temporary directory, plants one
mistake with a text substitution (a sign flip, a dropped term, an index slip,
a transposed operand, a dropped twiddle), compiles the copy with gcc and runs
a battery of the closed-form pins against it.  The unmodified source must pass
the battery and every mutant must fail it.  Nothing here touches a GPU.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "root_sign_flipped": ("*im = (double)sign * sin(angle);", "*im = -(double)sign * sin(angle);"),
    "naive_index_slip": ("int64_t e = (m * k) % N;", "int64_t e = (m * (k + 1)) % N;"),
    "naive_drops_last_term": ("for (int64_t k = 0; k < N; ++k) {\n            int64_t e",
                              "for (int64_t k = 0; k < N - 1; ++k) {\n            int64_t e"),
    "radix2_twiddle_off_by_one": ("root_of_unity(N, k, sign, &wr, &wi);",
                                  "root_of_unity(N, k + 1, sign, &wr, &wi);"),
    "radix2_sum_difference_swapped": ("y[2 * (k + h)] = er - tr;", "y[2 * (k + h)] = er + tr;"),
    "eq2_permutation_transposed": ("v[2 * (k * M + m)] = x[2 * (m * K + k)];",
                                   "v[2 * (k * M + m)] = x[2 * (k * M + m)];"),
    "eq2_twiddle_dropped": ("root_of_unity(N, k * j, sign, &wr, &wi);", "wr = 1.0; wi = 0.0;"),
    "eq2_twiddle_conjugated": ("root_of_unity(N, k * j, sign, &wr, &wi);",
                               "root_of_unity(N, k * j, -sign, &wr, &wi);"),
    "eq2_outer_dft_transposed": ("double zr = z[2 * (k * M + j1)], zi = z[2 * (k * M + j1) + 1];",
                                 "double zr = z[2 * (j1 * K + k)], zi = z[2 * (j1 * K + k) + 1];"),
    "eq2_outer_root_wrong_order": ("root_of_unity(K, j2 * k, sign, &wr, &wi);",
                                   "root_of_unity(N, j2 * k, sign, &wr, &wi);"),
}


def build_variant(tmp_path, name, subst):
    src = open(SRC).read()
    if subst is not None:
        old, new = subst
        assert src.count(old) >= 1, f"mutation {name}: pattern not found"
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", str(so), str(c), "-lm", "-lpthread"])
    lib = ctypes.CDLL(str(so))
    fns = {}
    for kind, sym in (("naive", "oracle_dft_naive"), ("radix2", "oracle_fft_radix2"),
                      ("eq2", "oracle_fft_eq2")):
        f = getattr(lib, sym)
        f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                      ctypes.c_int, ctypes.c_int]
        f.restype = ctypes.c_int

        def call(x, sign, f=f):
            x = np.ascontiguousarray(x, dtype=np.complex128).reshape(1, -1)
            y = np.empty_like(x)
            assert f(x.ctypes.data, y.ctypes.data, x.shape[1], 1, sign, 1) == 0
            return y[0]
        fns[kind] = call
    return fns


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def battery_passes(fns):
    """True iff every closed-form pin holds for every transform."""
    listing_x = np.array([1 + 1j, 2 + 2j, 3 + 3j, 4 + 4j])
    listing_y = np.array([10 + 10j, -4, -2 - 2j, -4j])
    a = 0.93 * np.exp(0.37j)
    for kind, f in fns.items():
        sizes = [4, 8, 16, 64] if kind == "radix2" else [4, 8, 12, 15, 16, 60, 64, 63]
        if np.max(np.abs(f(listing_x, -1) - listing_y)) > 1e-12:
            return False
        for n in sizes:
            k = np.arange(n)
            for sign in (-1, 1):
                want = (1 - a ** n) / (1 - a * np.exp(sign * 2j * np.pi * k / n))
                if rel(f(a ** k, sign), want) > 1e-12:
                    return False
                tone = np.zeros(n, complex)
                f0 = (3 * n) // 7 or 1
                tone[f0] = n
                if np.max(np.abs(f(np.exp(-sign * 2j * np.pi * f0 * k / n), sign) - tone)) > 1e-10:
                    return False
    return True


def test_unmodified_oracle_passes_battery(tmp_path):
    assert battery_passes(build_variant(tmp_path, "clean", None))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    assert not battery_passes(build_variant(tmp_path, name, MUTATIONS[name]))
