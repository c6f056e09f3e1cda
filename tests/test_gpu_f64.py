"""Complex128 path (FP64 arithmetic, the paper's own precision): parity with
the FP64 oracle through the C ABI, element by element on seeded inputs, for
every compiled FP64 variant and length, both directions; invariants; host
buffers; error codes."""
import math

import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED
F64_TOL_PER_LOG2N = 1e-15


def tol_f64(n):
    return F64_TOL_PER_LOG2N * max(1.0, math.log2(n))


def sizes():
    return [2 ** k for k in range(1, 13)] + [n for n in synth.size_family(3, 4096) if n & (n - 1)]


def reference(x, direction):
    # Eq. 2 recursion of the oracle: O(N log N), error ~ log2(N) * 2^-53
    return oracle.fft_eq2(np.asarray(x, np.complex128), direction, nthreads=ncpu())


def batch_c128(seed, n, batch):
    """complex128 rows: the float32 uniform generator widened, plus an exact
    low-order term so that the inputs use the full double significand."""
    x = synth.uniform_batch(seed, n, batch).astype(np.complex128)
    y = synth.uniform_batch(seed + 1, n, batch).astype(np.complex128)
    return x + y * 2.0 ** -26


def run(x, direction, variant=None, inplace=False):
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, n = x.shape
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.float64).reshape(-1)).cuda()
    d_out = d_in if inplace else torch.full_like(d_in, float("nan"))
    with gbfft.Plan(n, batch, direction, dtype=gbfft.GBFFT_C2C_F64, variant=variant) as p:
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
    return d_out.cpu().numpy().view(np.complex128).reshape(batch, n)


def check(y, x, direction):
    n = x.shape[1]
    err = row_rel_l2(y, reference(x, direction))
    assert np.all(np.isfinite(err)), "non-finite output"
    assert err.max() <= tol_f64(n), f"n={n} max rel-L2 {err.max():.3e} > {tol_f64(n):.3e}"
    return err


@pytest.mark.parametrize("direction", [-1, 1])
def test_every_f64_variant_every_size(direction):
    from paper_2207_06803_gb300 import gbfft
    worst = 0.0
    for n in sizes():
        v = 0
        while True:
            try:
                gbfft.Plan(n, 1, direction, dtype=gbfft.GBFFT_C2C_F64, variant=v).close()
            except gbfft.GbfftError as e:
                assert e.status == gbfft.GBFFT_ERR_NOT_FOUND and v > 0, (n, v)
                break
            batch = 3 * max(1, 1024 // n) + 1  # tiles hold at most 1024 elements: several CTAs, ragged tail
            x = batch_c128(SEED + n + v, n, batch)
            err = check(run(x, direction, variant=v), x, direction)
            worst = max(worst, float(err.max() / max(1.0, math.log2(n))))
            v += 1
    assert worst < F64_TOL_PER_LOG2N


@pytest.mark.parametrize("n", [8, 256, 4096, 96, 1792])
def test_f64_in_place_and_invariants(n):
    batch = 7
    x = batch_c128(SEED, n, batch)
    assert np.array_equal(run(x, -1), run(x, -1, inplace=True))
    delta = np.zeros((batch, n), np.complex128)
    delta[:, 0] = 1
    assert np.max(np.abs(run(delta, -1) - 1)) < 1e-15 * max(1, math.log2(n))
    c = np.full((batch, n), 0.5 - 0.25j)
    want = np.zeros((batch, n), np.complex128)
    want[:, 0] = n * (0.5 - 0.25j)
    assert np.max(np.abs(run(c, -1) - want)) < 1e-15 * n
    rt = run(run(x, -1), 1)
    assert row_rel_l2(rt, n * x).max() < 2 * tol_f64(n)


def test_f64_agrees_with_fp32_path_to_fp32_accuracy():
    from helpers import gpu_fft
    n, batch = 1024, 33
    x = batch_c128(SEED, n, batch)
    y64 = run(x, -1)
    y32 = gpu_fft(x.astype(np.complex64), -1)
    assert row_rel_l2(y32, y64).max() <= tol_fp32(n)


def test_f64_full_size_sampled_rows():
    """N = 4096 at batch 2^14 (1 GiB in, 1 GiB out), 256 seeded rows vs the oracle."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    n, batch = 4096, 1 << 14
    flat = synth.uniform_flat(SEED, 0, n * batch).astype(np.complex128)
    d_in = torch.from_numpy(flat.view(np.float64)).cuda()
    d_out = torch.empty_like(d_in)
    with gbfft.Plan(n, batch, -1, dtype=gbfft.GBFFT_C2C_F64) as p:
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
    rows = synth.sample_rows(SEED, batch, 256)
    y = d_out.view(batch, 2 * n)[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.complex128)
    check(y, flat.reshape(batch, n)[rows], -1)


def test_f64_host_buffers():
    from paper_2207_06803_gb300 import gbfft
    n, batch = 512, 3000
    x = batch_c128(SEED + 5, n, batch)
    y = np.empty_like(x)
    with gbfft.Plan(n, batch, -1, dtype=gbfft.GBFFT_C2C_F64) as p:
        gbfft.gbfft_execute_host(p.handle, x.ctypes.data, y.ctypes.data)
    check(y, x, -1)


def test_f64_error_codes():
    from paper_2207_06803_gb300 import gbfft
    for bad in (8192, 11, 9, 15 * 16):  # too long; prime 11; two odd factors
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_plan_create(bad, 4, -1, gbfft.GBFFT_C2C_F64)
        assert e.value.status == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create_twopass(4096, 4, -1, gbfft.GBFFT_C2C_F64, 64)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_ragged([16, 32], [0, 16], -1, gbfft.GBFFT_C2C_F64)
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
