"""Multi-dimensional transforms DFT_{d0} ⊗ ... ⊗ DFT_{d(r-1)} (Table I's Kronecker
product applied to whole transforms) through the C ABI, against the oracle's
``dft_nd`` (pinned to the direct multi-dimensional DFT sum in
``test_oracle_pins.py``)."""
import math

import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

SEED = synth.DEFAULT_SEED


def run_nd(x, direction, inplace=False):
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, dims = x.shape[0], x.shape[1:]
    d_in = torch.from_numpy(np.ascontiguousarray(x, np.complex64).view(np.float32).reshape(-1)).cuda()
    d_out = d_in if inplace else torch.full_like(d_in, float("nan"))
    with gbfft.Plan(tuple(dims), batch, direction) as p:
        assert gbfft.gbfft_plan_dims(p.handle) == list(dims)
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
    return d_out.cpu().numpy().view(np.complex64).reshape(x.shape)


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(8, 16), (16, 64), (32, 256), (96, 48), (512, 1024), (128, 4096),
                                  (8, 16, 32), (16, 32, 64), (32, 32, 32), (64, 8, 1536)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_nd_matches_the_oracle(dims, direction):
    total = math.prod(dims)
    batch = max(1, min(3, (1 << 22) // total))
    x = synth.uniform_flat(SEED + total, 0, batch * total).reshape((batch,) + dims)
    y = run_nd(x, direction)
    ref = oracle.dft_nd(x, direction, nthreads=ncpu())
    err = row_rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))
    tol = sum(tol_fp32(d) for d in dims)  # one FP32 transform per axis
    assert np.all(np.isfinite(err)) and err.max() <= tol, (dims, err.max(), tol)


@pytest.mark.gpu
def test_nd_in_place_and_host_buffers():
    from paper_2207_06803_gb300 import gbfft
    dims, batch = (64, 128), 5
    x = synth.uniform_flat(SEED, 0, batch * 64 * 128).reshape((batch,) + dims)
    a = run_nd(x, -1)
    b = run_nd(x, -1, inplace=True)
    assert np.array_equal(a, b)
    h = np.empty_like(x)
    with gbfft.Plan(dims, batch, -1) as p:
        gbfft.gbfft_execute_host(p.handle, x.ctypes.data, h.ctypes.data)
    assert np.array_equal(h, a)


@pytest.mark.gpu
def test_nd_errors():
    from paper_2207_06803_gb300 import gbfft
    for dims in [(8, 8), (7, 16), (16, 8192), (1000, 16)]:
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_plan_create_nd(dims, 2)
        assert e.value.status == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE, dims
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create_nd((8, 8, 8, 16), 2)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create_nd((8, 16), 2, -1, gbfft.GBFFT_C2C_F64)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
