"""Planner wisdom files: parsing, GPU-name filtering and lookup run on the
host (no device needed); malformed files are rejected."""
import pytest

from paper_2207_06803_gb300 import gbfft


@pytest.fixture(autouse=True)
def clean_table():
    gbfft.gbfft_wisdom_forget()
    yield
    gbfft.gbfft_wisdom_forget()


def test_import_lookup_forget(tmp_path):
    f = tmp_path / "w.txt"
    f.write_text("gbfft-wisdom 1 Some_GPU 4096 0 -1 2 0 0.162000\n"
                 "gbfft-wisdom 1 Some_GPU 8192 0 -1 -1 64 0.320000\n"
                 "gbfft-wisdom 1 Some_GPU 256 1 1 1 0 0.110000\n")
    gbfft.gbfft_wisdom_import(str(f), require_same_gpu=False)
    assert gbfft.gbfft_wisdom_lookup(4096, 0, -1) == (2, 0)
    assert gbfft.gbfft_wisdom_lookup(8192, 0, -1) == (-1, 64)
    assert gbfft.gbfft_wisdom_lookup(256, 1, 1) == (1, 0)
    assert gbfft.gbfft_wisdom_lookup(4096, 0, 1) is None
    gbfft.gbfft_wisdom_forget()
    assert gbfft.gbfft_wisdom_lookup(4096, 0, -1) is None


def test_other_gpu_entries_are_skipped(tmp_path):
    f = tmp_path / "w.txt"
    f.write_text("gbfft-wisdom 1 Not_This_GPU_XYZ 4096 0 -1 2 0 0.162000\n")
    gbfft.gbfft_wisdom_import(str(f), require_same_gpu=True)
    assert gbfft.gbfft_wisdom_lookup(4096, 0, -1) is None


def test_malformed_and_missing_files(tmp_path):
    f = tmp_path / "bad.txt"
    f.write_text("this is not wisdom\n")
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_wisdom_import(str(f), require_same_gpu=False)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_wisdom_import(str(tmp_path / "missing.txt"), require_same_gpu=False)
    assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND
