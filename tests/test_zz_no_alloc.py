"""The allocation-free two-pass entry point.

Some callers cannot allocate device memory when they transform: hosts that
own all device memory through a fixed arena of their own, or real-time loops
that must not allocate after start-up.  gbfft_execute_twopass_noalloc serves
them from a static device array inside the library.  This checks, through
the C ABI, that two calls in a row give the same result as the regular
two-pass plan (the entry point that allocates its workspace) and as the FP64
oracle, within the FP32 tolerance the other tests use; that an in-place call
gives the same result; and that the argument checks return their codes.  The
file sorts last so that a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import gbfft, synth

pytestmark = pytest.mark.gpu


def _noalloc(lib, n, batch, direction, d_in, d_out, stream_handle):
    return lib.gbfft_execute_twopass_noalloc(ctypes.c_int64(n), ctypes.c_int64(batch), direction,
                                             ctypes.c_void_p(d_in), ctypes.c_void_p(d_out),
                                             ctypes.c_void_p(stream_handle))


@pytest.mark.parametrize("n,batch,direction", [(8192, 96, -1), (16384, 40, 1), (6144, 33, -1)])
def test_noalloc_matches_twopass_plan_on_two_calls(n, batch, direction):
    import torch
    lib = gbfft.lib()
    xs = [synth.uniform_batch(synth.DEFAULT_SEED + i, n, batch) for i in range(2)]
    stream = torch.cuda.current_stream()
    for x in xs:  # two calls in a row share the static array
        d_in = torch.from_numpy(x.view(np.float32).reshape(-1)).cuda()
        d_ref = torch.empty_like(d_in)
        d_out = torch.full_like(d_in, float("nan"))
        with gbfft.Plan(n, batch, direction, k_outer=0) as p:
            p.execute(d_in, d_ref, stream)
        rc = _noalloc(lib, n, batch, direction, d_in.data_ptr(), d_out.data_ptr(), stream.cuda_stream)
        assert rc == gbfft.GBFFT_OK
        torch.cuda.synchronize()
        y = d_out.cpu().numpy().view(np.complex64).reshape(batch, n)
        ref = d_ref.cpu().numpy().view(np.complex64).reshape(batch, n)
        assert np.all(np.isfinite(y))
        assert row_rel_l2(y, ref).max() <= tol_fp32(n)
        # and against the oracle itself, on a seeded sample of rows
        rows = synth.sample_rows(synth.DEFAULT_SEED, batch, 8)
        want = oracle.dft(x[rows].astype(np.complex128), direction, nthreads=ncpu())
        assert row_rel_l2(y[rows], want).max() <= tol_fp32(n)


def test_noalloc_in_place_equals_out_of_place():
    import torch
    lib = gbfft.lib()
    n, batch = 10240, 24
    x = synth.uniform_batch(synth.DEFAULT_SEED + 5, n, batch)
    stream = torch.cuda.current_stream()
    d_a = torch.from_numpy(x.view(np.float32).reshape(-1)).cuda()
    d_oop = torch.full_like(d_a, float("nan"))
    assert _noalloc(lib, n, batch, -1, d_a.data_ptr(), d_oop.data_ptr(), stream.cuda_stream) == gbfft.GBFFT_OK
    assert _noalloc(lib, n, batch, -1, d_a.data_ptr(), d_a.data_ptr(), stream.cuda_stream) == gbfft.GBFFT_OK
    torch.cuda.synchronize()
    assert torch.equal(d_a, d_oop)
    want = oracle.dft(x[:4].astype(np.complex128), -1, nthreads=ncpu())
    y = d_a.cpu().numpy().view(np.complex64).reshape(batch, n)
    assert row_rel_l2(y[:4], want).max() <= tol_fp32(n)


def test_noalloc_rejects_sizes_beyond_the_static_array():
    import torch
    lib = gbfft.lib()
    d = torch.empty(16, device="cuda")
    for n, batch in ((8192, 1024),          # 64 MiB of workspace alone: over the limit
                     (8192, 1 << 60)):      # a byte count that would wrap 64 bits
        rc = _noalloc(lib, n, batch, -1, d.data_ptr(), d.data_ptr(), 0)
        assert rc == gbfft.GBFFT_ERR_BUDGET


def test_noalloc_argument_checks():
    import torch
    lib = gbfft.lib()
    n, batch = 8192, 2
    d = torch.zeros(2 * n * batch * 2 + 64, device="cuda")
    base = d.data_ptr()
    # a pointer off the 16-byte grid
    assert _noalloc(lib, n, batch, -1, base + 8, base + 2 * 8 * n * batch + 64, 0) == gbfft.GBFFT_ERR_ALIGNMENT
    # output overlapping the input without being the same buffer
    assert _noalloc(lib, n, batch, -1, base, base + 8 * n, 0) == gbfft.GBFFT_ERR_OVERLAP
    # a length with a prime factor above 7
    assert _noalloc(lib, 11 * 1024, 1, -1, base, base, 0) == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
    assert _noalloc(lib, n, batch, 3, base, base, 0) == gbfft.GBFFT_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.count_nonzero(d).item() == 0  # no rejected call wrote anything
