"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/*.h declares; host-side argument checks run without
touching a device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2207_06803_gb300 import gbfft

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(gbfft_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return gbfft.lib()


def test_header_declares_functions():
    names = declared_functions()
    assert "gbfft_plan_create" in names and "gbfft_execute" in names and "gbfft_destroy" in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(gbfft.PROTOTYPES)
    for name in gbfft.PROTOTYPES:
        assert hasattr(gbfft, name), name


def test_status_strings(lib):
    for code in range(0, 11):
        s = gbfft.gbfft_status_string(code)
        assert s and s != "unknown status"
    assert gbfft.gbfft_status_string(99) == "unknown status"


def test_host_side_argument_checks_need_no_device(lib):
    h = ctypes.c_void_p()
    assert lib.gbfft_plan_create(None, 64, 1, -1, 0) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_plan_create(ctypes.byref(h), 0, 1, -1, 0) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_plan_create(ctypes.byref(h), 64, -1, -1, 0) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_plan_create(ctypes.byref(h), 64, 1, 2, 0) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_plan_create(ctypes.byref(h), 64, 1, -1, 77) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_plan_create(ctypes.byref(h), 11, 1, -1, 0) == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
    assert lib.gbfft_plan_create(ctypes.byref(h), 13 * 64, 1, -1, 0) == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
    assert h.value is None
    assert lib.gbfft_execute(None, None, None, None) == gbfft.GBFFT_ERR_INVALID_ARG
    assert lib.gbfft_destroy(None) == gbfft.GBFFT_OK


def test_variant_registry_is_consistent(lib):
    from paper_2207_06803_gb300 import synth
    sizes = [2 ** k for k in range(1, 13)] + [n for n in synth.size_family(3, 4096) if n & (n - 1)]
    for n in sizes:
        nv = gbfft.gbfft_num_variants(n)
        assert nv >= 1, n
        for i in range(nv):
            info = gbfft.gbfft_variant_info(n, i)
            prod = 1
            for r in info["radices"]:
                assert r in (2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64)
                prod *= r
            assert prod == n
            assert info["threads_per_cta"] * (n * info["rows_per_cta"] // info["threads_per_cta"]) \
                == n * info["rows_per_cta"]
            assert info["threads_per_cta"] <= 1024 and info["smem_bytes"] <= 227 * 1024
        with pytest.raises(gbfft.GbfftError):
            gbfft.gbfft_variant_info(n, nv)
