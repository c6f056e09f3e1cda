"""Parity of the single-pass Stockham kernels with the FP64 oracle, through the
C ABI, element by element on seeded inputs; plus invariants, edge cases and
guard bands around the output."""
import math

import numpy as np
import pytest

import oracle
from helpers import gpu_fft, ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED


def single_pass_sizes():
    return [2 ** k for k in range(1, 13)] + [n for n in synth.size_family(3, 4096) if n & (n - 1)]


def reference(x, direction):
    return oracle.dft(x.astype(np.complex128), direction, nthreads=ncpu())


def check(y, x, direction, tol=None):
    n = x.shape[1]
    err = row_rel_l2(y, reference(x, direction))
    tol = tol_fp32(n) if tol is None else tol
    assert np.all(np.isfinite(err)), "non-finite output"
    assert err.max() <= tol, f"n={n} max rel-L2 {err.max():.3e} > {tol:.3e}"
    return err


def test_pr1_forward_n64_batch4096_all_rows():
    n, batch = 64, 4096
    x = synth.uniform_batch(SEED, n, batch)
    y = gpu_fft(x, -1)
    err = check(y, x, -1)
    # the paper's own metric (Sec. VI): max |y - y_ref| / N, reported beside the gate
    ref = reference(x, -1)
    assert np.max(np.abs(y - ref)) / n < 1e-6
    assert err.mean() < 1e-7


@pytest.mark.parametrize("direction", [-1, 1])
def test_every_variant_every_size(direction):
    from paper_2207_06803_gb300 import gbfft
    for n in single_pass_sizes():
        for v in range(gbfft.gbfft_num_variants(n)):
            rows = gbfft.gbfft_variant_info(n, v)["rows_per_cta"]
            batch = 3 * rows + 1  # several CTAs and a ragged last tile
            x = synth.uniform_batch(SEED + n + v, n, batch)
            check(gpu_fft(x, direction, variant=v), x, direction)


def test_persistent_variants_walk_many_tiles():
    """Persistent kernels (register prefetch, TMA bulk-copy prefetch) over
    enough rows that every CTA walks several tiles, plus a ragged last tile:
    bit-identical to the one-tile-per-CTA kernel with the same schedule, and
    within tolerance of the oracle on sampled rows."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    checked = 0
    for n in single_pass_sizes():
        kinds = [gbfft.gbfft_variant_kind(n, v) for v in range(gbfft.gbfft_num_variants(n))]
        for v, kind in enumerate(kinds):
            if kind not in (1, 3):
                continue
            rad = gbfft.gbfft_variant_info(n, v)["radices"]
            ref_v = next((w for w, k in enumerate(kinds) if k == 0 and gbfft.gbfft_variant_info(n, w)["radices"] == rad), None)
            batch = (1 << 23) // n + 3
            x = synth.uniform_batch(SEED + v, n, batch)
            d_in = torch.from_numpy(x.view(np.float32).reshape(-1)).cuda()
            outs = []
            for var in ([v] if ref_v is None else [v, ref_v]):
                d_out = torch.full_like(d_in, float("nan"))
                with gbfft.Plan(n, batch, -1, variant=var) as p:
                    p.execute(d_in, d_out)
                    torch.cuda.synchronize()
                    assert gbfft.gbfft_plan_device_status(p.handle) == 0
                outs.append(d_out)
            if len(outs) == 2:
                assert torch.equal(outs[0], outs[1]), (n, v, ref_v)
            rows = synth.sample_rows(SEED, batch, 64)
            rows = np.concatenate([rows, [batch - 1]])
            y = outs[0].view(batch, 2 * n)[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.complex64)
            check(y, x[rows], -1)
            checked += 1
    assert checked >= 4


@pytest.mark.parametrize("n", [8, 64, 256, 1024, 4096, 96, 640, 3584])
def test_in_place_equals_out_of_place(n):
    x = synth.uniform_batch(SEED, n, 37)
    a = gpu_fft(x, -1)
    b = gpu_fft(x, -1, inplace=True)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n", [2, 16, 64, 512, 4096, 12, 320, 1792])
def test_invariants_on_gpu(n):
    batch = 5
    delta = np.zeros((batch, n), np.complex64)
    delta[:, 0] = 1
    y = gpu_fft(delta, -1)
    assert np.max(np.abs(y - 1)) < 1e-6
    c = np.full((batch, n), 0.5 - 0.25j, np.complex64)
    y = gpu_fft(c, -1)
    want = np.zeros((batch, n), np.complex128)
    want[:, 0] = n * (0.5 - 0.25j)
    assert np.max(np.abs(y - want)) < 1e-6 * n
    x = synth.uniform_batch(SEED, n, batch)
    rt = gpu_fft(gpu_fft(x, -1), 1)
    assert row_rel_l2(rt, n * x.astype(np.complex128)).max() < 2 * tol_fp32(n)


def test_batch_one_and_zero():
    from paper_2207_06803_gb300 import gbfft
    import torch
    x = synth.uniform_batch(SEED, 256, 1)
    check(gpu_fft(x, -1), x, -1)
    d = torch.zeros(16, device="cuda")
    with gbfft.Plan(256, 0) as p:
        p.execute(d, d)  # no-op


def test_error_codes():
    import torch
    from paper_2207_06803_gb300 import gbfft
    buf = torch.zeros(2 * 64 * 8 + 64, device="cuda")
    with gbfft.Plan(64, 8) as p:
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_execute(p.handle, buf.data_ptr() + 4, buf.data_ptr() + 4096 + 256)
        assert e.value.status == gbfft.GBFFT_ERR_ALIGNMENT
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_execute(p.handle, buf.data_ptr(), buf.data_ptr() + 16)
        assert e.value.status == gbfft.GBFFT_ERR_OVERLAP
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_execute(p.handle, 0, buf.data_ptr())
        assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    for n in (11, 13 * 64, 0):
        with pytest.raises(gbfft.GbfftError):
            gbfft.gbfft_plan_create(n, 4)
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_create_variant(64, 4, -1, 0, 99)
    assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND


@pytest.mark.parametrize("n", [8, 128, 4096, 1536])
def test_guard_bands_untouched(n):
    """Canary words before and after the output stay intact (stands in for a
    memory checker)."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    batch, guard = 19, 1024  # guard in float32 words
    x = synth.uniform_batch(SEED, n, batch)
    d_in = torch.from_numpy(x.view(np.float32).reshape(-1)).cuda()
    canary = float.fromhex("0x1.dead0p+100")
    big = torch.full((2 * guard + 2 * n * batch,), canary, device="cuda")
    out = big[guard: guard + 2 * n * batch]
    with gbfft.Plan(n, batch) as p:
        p.execute(d_in, out)
    torch.cuda.synchronize()
    assert torch.all(big[:guard] == canary) and torch.all(big[guard + 2 * n * batch:] == canary)
    check(out.cpu().numpy().view(np.complex64).reshape(batch, n), x, -1)


@pytest.mark.parametrize("direction", [-1, 1])
def test_full_size_sweep_sampled_rows(direction):
    """N = 2^3..2^12 at batch 2^26/N (512 MiB per call), 1024 seeded rows per
    size against the oracle."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    total = 1 << 26
    flat = synth.uniform_flat(SEED, 0, total)
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    d_out = torch.empty_like(d_in)
    for k in range(3, 13):
        n = 1 << k
        batch = total // n
        with gbfft.Plan(n, batch, direction) as p:
            p.execute(d_in, d_out)
            torch.cuda.synchronize()
        rows = synth.sample_rows(SEED + k, batch, 1024)
        idx = torch.from_numpy(rows).cuda()
        y = d_out.view(batch, 2 * n).index_select(0, idx).cpu().numpy().view(np.complex64)
        x = flat.reshape(batch, n)[rows]
        check(y, x, direction)


def test_autotune_records_wisdom_that_plans_use(tmp_path):
    from paper_2207_06803_gb300 import gbfft
    gbfft.gbfft_wisdom_forget()
    try:
        for n in (1024, 4096, 8192):
            best = gbfft.gbfft_autotune(n, (1 << 22) // n, -1, 0, reps=3)
            assert best["ms"] > 0
            assert gbfft.gbfft_wisdom_lookup(n, 0, -1) == (best["variant"], best["k_outer"])
            with gbfft.Plan(n, 8, -1) as p:
                info = p.info()
                if best["k_outer"] > 0:
                    assert info["k_outer"] == best["k_outer"]
                else:
                    assert info["variant"] == best["variant"]
        path = tmp_path / "wisdom.txt"
        gbfft.gbfft_wisdom_export(str(path))
        gbfft.gbfft_wisdom_forget()
        gbfft.gbfft_wisdom_import(str(path), require_same_gpu=True)
        assert gbfft.gbfft_wisdom_lookup(4096, 0, -1) is not None
        x = synth.uniform_batch(SEED, 4096, 9)
        check(gpu_fft(x, -1), x, -1)  # a wisdom-driven plan still matches the oracle
    finally:
        gbfft.gbfft_wisdom_forget()


@pytest.mark.parametrize("direction", [-1, 1])
def test_pease_variants_at_scale(direction):
    """Pease's constant-geometry kernels (variant kind 5) over 2^22 points plus
    a ragged last tile, sampled rows and the last row against the oracle; the
    guard band past the output stays untouched."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    covered = []
    for n in single_pass_sizes():
        for v in range(gbfft.gbfft_num_variants(n)):
            if gbfft.gbfft_variant_kind(n, v) != 5:
                continue
            rows = gbfft.gbfft_variant_info(n, v)["rows_per_cta"]
            batch = (1 << 22) // n + rows // 2 + 1
            x = synth.uniform_batch(SEED + 5 * n, n, batch)
            d_in = torch.from_numpy(x.view(np.float32).reshape(-1)).cuda()
            d_out = torch.full((2 * n * batch + 64,), float("nan"), device="cuda")
            with gbfft.Plan(n, batch, direction, variant=v) as p:
                p.execute(d_in, d_out[: 2 * n * batch])
                torch.cuda.synchronize()
                assert gbfft.gbfft_plan_device_status(p.handle) == 0
            assert torch.isnan(d_out[2 * n * batch:]).all()
            pick = np.concatenate([synth.sample_rows(SEED, batch, 48), [batch - 1]])
            y = d_out[: 2 * n * batch].view(batch, 2 * n)[torch.from_numpy(pick).cuda()].cpu().numpy()
            check(y.view(np.complex64), x[pick], direction)
            covered.append(n)
    assert sorted(covered) == [64, 256, 512, 4096]
