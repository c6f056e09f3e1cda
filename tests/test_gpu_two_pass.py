"""Parity of the two-pass Eq. 2 path (column transforms + D^N_M + column
transforms) with the FP64 oracle, and of the host-buffer pipeline with the
device-buffer call."""
import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED


def run(x, direction=-1, k_outer=None, inplace=False):
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, n = x.shape
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.float32).reshape(-1)).cuda()
    d_out = d_in if inplace else torch.empty_like(d_in)
    with gbfft.Plan(n, batch, direction, k_outer=k_outer) as p:
        info = p.info()
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.complex64).reshape(batch, n), info


def check(y, x, direction):
    n = x.shape[1]
    ref = oracle.dft(x.astype(np.complex128), direction, nthreads=ncpu())
    err = row_rel_l2(y, ref)
    assert err.max() <= tol_fp32(n), f"n={n} max rel-L2 {err.max():.3e} > {tol_fp32(n):.3e}"


@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("n", [5120, 6144, 7168, 8192, 10240, 12288, 14336, 16384])
def test_long_family_sizes_two_pass_plan(n, direction):
    x = synth.uniform_batch(SEED + n, n, 3)
    y, info = run(x, direction, k_outer=0)  # the two-pass form with the planner's split
    assert info["k_outer"] * info["m_inner"] == n and info["k_outer"] > 1
    assert info["workspace_bytes"] == 8 * n * 3
    check(y, x, direction)


@pytest.mark.parametrize("n,k", [(1024, 32), (4096, 32), (4096, 64), (4096, 128), (2048, 64),
                                 (96 * 128, 96), (48 * 80, 48), (112 * 112, 112), (512 * 32, 32)])
def test_forced_splits(n, k):
    x = synth.uniform_batch(SEED + n + k, n, 5)
    y, info = run(x, -1, k_outer=k)
    assert (info["k_outer"], info["m_inner"]) == (k, n // k)
    check(y, x, -1)


@pytest.mark.parametrize("n", [32768, 65536, 262144])
def test_beyond_single_pass_range(n):
    x = synth.uniform_batch(SEED, n, 2)
    y, _ = run(x, -1)
    check(y, x, -1)


def test_two_pass_in_place():
    x = synth.uniform_batch(SEED, 8192, 7)
    a, _ = run(x, -1, k_outer=0)
    b, _ = run(x, -1, k_outer=0, inplace=True)
    assert np.array_equal(a, b)


def test_unsupported_splits():
    from paper_2207_06803_gb300 import gbfft
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create_twopass(8192, 2, -1, 0, 3)
    assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create(13 * 1024, 2)
    assert e.value.status == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE


@pytest.mark.parametrize("n", [8192, 16384])
def test_full_size_sampled_rows(n):
    """512 MiB per call (batch 2^26/N) plus an equal workspace; 256 seeded rows."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    total = 1 << 26
    batch = total // n
    flat = synth.uniform_flat(SEED, 0, total)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    with gbfft.Plan(n, batch, -1, k_outer=0) as p:  # Eq. 2 as two passes, the planner's split
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
    rows = synth.sample_rows(SEED + n, batch, 256)
    y = d_out.view(batch, 2 * n).index_select(0, torch.from_numpy(rows).cuda()).cpu().numpy().view(np.complex64)
    check(y, flat.reshape(batch, n)[rows], -1)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,batch,kwargs", [(4096, 2500, {}), (64, 300000, {}), (8192, 1100, {}),
                                            (1000 * 0 + 4096, 2100, {"k_outer": 64})])
def test_host_pipeline_matches_device_call(n, batch, kwargs, pinned):
    """gbfft_execute_host on page-locked buffers runs the kernels on them
    directly (the device addresses them); on pageable buffers it streams the
    batch through the staging ring in 32 MiB chunks.  Either way its result
    equals the device-buffer call bit for bit."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    x = synth.uniform_batch(SEED, n, batch)
    h_in = torch.from_numpy(x.view(np.float32).reshape(-1))
    h_out = torch.empty_like(h_in)
    if pinned:
        h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
    d_in = h_in.cuda()
    d_out = torch.empty_like(d_in)
    with gbfft.Plan(n, batch, -1, **kwargs) as p:
        p.execute(d_in, d_out)
        p.execute_host(h_in, h_out)
        p.execute_host(h_in, h_out)  # reuse of the ring
        torch.cuda.synchronize()
    assert torch.equal(h_out, d_out.cpu())
    rows = np.array([0, batch // 2, batch - 1])
    check(h_out.numpy().view(np.complex64).reshape(batch, n)[rows], x[rows], -1)
