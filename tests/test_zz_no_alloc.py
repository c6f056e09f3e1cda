"""The allocation-free two-pass entry point.

Some callers cannot allocate device memory when they transform: hosts that
own all device memory through a fixed arena of their own, or real-time loops
that must not allocate after start-up.  gbfft_execute_twopass_noalloc serves
them from a static device array inside the library.  This checks, through
the C ABI, that two calls in a row give the same result as the regular
two-pass plan (the entry point that allocates its workspace), within the
FP32 tolerance the other tests use.  The file sorts last so that a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from helpers import row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import gbfft, synth

pytestmark = pytest.mark.gpu


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
        rc = lib.gbfft_execute_twopass_noalloc(ctypes.c_int64(n), ctypes.c_int64(batch), direction,
                                               ctypes.c_void_p(d_in.data_ptr()), ctypes.c_void_p(d_out.data_ptr()),
                                               ctypes.c_void_p(stream.cuda_stream))
        assert rc == gbfft.GBFFT_OK
        torch.cuda.synchronize()
        y = d_out.cpu().numpy().view(np.complex64).reshape(batch, n)
        ref = d_ref.cpu().numpy().view(np.complex64).reshape(batch, n)
        assert np.all(np.isfinite(y))
        assert row_rel_l2(y, ref).max() <= tol_fp32(n)


def test_noalloc_rejects_sizes_beyond_the_static_array():
    import torch
    lib = gbfft.lib()
    n, batch = 8192, 1024  # 64 MiB of workspace alone: over the limit
    d = torch.empty(16, device="cuda")
    rc = lib.gbfft_execute_twopass_noalloc(ctypes.c_int64(n), ctypes.c_int64(batch), -1,
                                           ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(d.data_ptr()),
                                           ctypes.c_void_p(0))
    assert rc == gbfft.GBFFT_ERR_BUDGET
