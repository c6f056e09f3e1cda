"""One-pass transforms for 4096 < N <= 32768 on thread-block clusters (Eq. 2
with the row kept on chip): every compiled cluster variant against the FP64
oracle, both directions, several rows; in place; agreement with the two-pass
form (the default for these lengths); sampled rows at full size."""
import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED
CLUSTER_SIZES = [5120, 6144, 7168, 8192, 10240, 12288, 14336, 16384, 20480, 24576, 28672, 32768]


def run(x, direction, variant=None, k_outer=None, inplace=False):
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, n = x.shape
    d_in = torch.from_numpy(np.ascontiguousarray(x).view(np.float32).reshape(-1)).cuda()
    d_out = d_in if inplace else torch.full_like(d_in, float("nan"))
    with gbfft.Plan(n, batch, direction, variant=variant, k_outer=k_outer) as p:
        info = p.info()
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
    return d_out.cpu().numpy().view(np.complex64).reshape(batch, n), info


def check(y, x, direction):
    n = x.shape[1]
    err = row_rel_l2(y, oracle.dft(x.astype(np.complex128), direction, nthreads=ncpu()))
    assert np.all(np.isfinite(err)) and err.max() <= tol_fp32(n), (n, err.max())


@pytest.mark.parametrize("direction", [-1, 1])
def test_every_cluster_variant(direction):
    from paper_2207_06803_gb300 import gbfft
    for n in CLUSTER_SIZES:
        nv = gbfft.gbfft_num_variants(n)
        assert nv >= 1
        for v in range(nv):
            assert gbfft.gbfft_variant_kind(n, v) == 4
            rad = gbfft.gbfft_variant_info(n, v)["radices"]
            assert int(np.prod(rad)) == n
            x = synth.uniform_batch(SEED + n + v, n, 3)
            y, info = run(x, direction, variant=v)
            assert info["radices"] == rad
            check(y, x, direction)


@pytest.mark.parametrize("n", [8192, 12288, 32768])
def test_cluster_in_place_and_two_pass_agree(n):
    x = synth.uniform_batch(SEED, n, 5)
    a, info = run(x, -1, variant=0)
    assert info["k_outer"] == 1 and info["workspace_bytes"] == 0  # one pass, no workspace
    b, _ = run(x, -1, variant=0, inplace=True)
    assert np.array_equal(a, b)
    c, info2 = run(x, -1, k_outer=0)  # Eq. 2 as two passes with the planner's split
    assert info2["k_outer"] > 1
    assert row_rel_l2(a, c).max() <= 2 * tol_fp32(n)


@pytest.mark.parametrize("n", [8192, 32768])
def test_cluster_full_size_sampled_rows(n):
    import torch
    from paper_2207_06803_gb300 import gbfft
    total = 1 << 26
    batch = total // n
    flat = synth.uniform_flat(SEED, 0, total)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    with gbfft.Plan(n, batch, -1, variant=0) as p:
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
    rows = np.concatenate([synth.sample_rows(SEED, batch, 64), [batch - 1]])
    y = d_out.view(batch, 2 * n)[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.complex64)
    check(y, flat.reshape(batch, n)[rows], -1)


def test_default_plan_above_4096():
    """The cluster kernel is the default where it measured faster (N = 5120,
    6144, 7168, 8192, 10240); other lengths above 4096 default to Eq. 2 as two
    passes."""
    from paper_2207_06803_gb300 import gbfft
    for n, one_pass in ((8192, True), (5120, True), (6144, True), (7168, True), (10240, True), (12288, False),
                        (14336, False), (16384, False), (65536, False)):
        with gbfft.Plan(n, 4, -1) as p:
            k, _ = gbfft.gbfft_plan_factors(p.handle)
            assert (k == 1) == one_pass, (n, k)
            if one_pass:
                assert gbfft.gbfft_variant_kind(n, p.info()["variant"]) == 4
