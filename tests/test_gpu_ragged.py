"""Ragged batches: one persistent launch (replayed from a CUDA graph) over
transforms of 41 different lengths (and of any length n <= 8192 whose prime
factors are 2, 3, 5, 7), checked transform by transform against
the FP64 oracle; tile-shape autotuning; buffer patching; failure injection
with a bounded wait."""
import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED


def ragged_case(count, seed=SEED):
    sizes = synth.ragged_sizes(seed, count)
    offs = synth.ragged_offsets(sizes)
    total = int(offs[-1] + sizes[-1])
    flat = synth.uniform_flat(seed, 0, total)
    return sizes, offs, flat


def check_all(y_flat, x_flat, sizes, offs, direction=-1, skip=()):
    """Every transform against the oracle, grouped by length."""
    by_n = {}
    for i, (n, o) in enumerate(zip(sizes.tolist(), offs.tolist())):
        if i not in skip:
            by_n.setdefault(n, []).append(o)
    for n, starts in by_n.items():
        idx = np.asarray(starts)[:, None] + np.arange(n)[None, :]
        x = x_flat[idx].astype(np.complex128)
        ref = oracle.dft(x, direction, nthreads=ncpu())
        err = row_rel_l2(y_flat[idx], ref)
        assert np.all(np.isfinite(err)), n
        assert err.max() <= tol_fp32(n), f"n={n} max rel-L2 {err.max():.3e}"


def run_plan(plan, flat, d_out=None):
    import torch
    d_in = torch.from_numpy(flat.view(np.float32)).cuda()
    if d_out is None:
        d_out = torch.full_like(d_in, float("nan"))
    plan.execute(d_in, d_out)
    torch.cuda.synchronize()
    return d_in, d_out


def to_np(t):
    return t.cpu().numpy().view(np.complex64)


@pytest.mark.parametrize("engine", ["compiled", "runtime"])
@pytest.mark.parametrize("direction", [-1, 1])
def test_ragged_10000_transforms_41_sizes(direction, engine):
    """Every one of the 41 family lengths has a compiled schedule (the
    default); the same plan switched to the run-time engine must agree with the
    oracle too."""
    from paper_2207_06803_gb300 import gbfft
    sizes, offs, flat = ragged_case(10000)
    assert len(set(sizes.tolist())) == 41
    with gbfft.RaggedPlan(sizes, offs, direction) as p:
        assert all(gbfft.gbfft_ragged_engine(p.handle, n) == 1 for n in set(sizes.tolist()))
        if engine == "runtime":
            gbfft.gbfft_ragged_set_engine(p.handle, 0, 0)
            assert all(gbfft.gbfft_ragged_engine(p.handle, n) == 0 for n in set(sizes.tolist()))
        assert p.num_items() > 0
        _, d_out = run_plan(p, flat)
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
        y = to_np(d_out)
    check_all(y, flat, sizes, offs, direction)


def test_ragged_queue_orders_agree():
    """The three queue orders (one queue by item work; one queue grouped by
    length; one sub-queue per length with home sub-queues per SM and stealing)
    only change which CTA runs which item: outputs are bit-identical and match
    the oracle, and an invalid order is refused."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    sizes, offs, flat = ragged_case(3000, seed=SEED + 5)
    outs = []
    with gbfft.RaggedPlan(sizes, offs) as p:
        assert gbfft.gbfft_ragged_queue_order(p.handle) == 1
        for order in (0, 1, 2):
            gbfft.gbfft_ragged_set_queue_order(p.handle, order)
            assert gbfft.gbfft_ragged_queue_order(p.handle) == order
            _, d_out = run_plan(p, flat)
            assert gbfft.gbfft_plan_device_status(p.handle) == 0
            outs.append(d_out)
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_ragged_set_queue_order(p.handle, 3)
        assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
    check_all(to_np(outs[2]), flat, sizes, offs)


def test_ragged_in_place_and_buffer_patching():
    import torch
    from paper_2207_06803_gb300 import gbfft
    sizes, offs, flat = ragged_case(600, seed=SEED + 1)
    with gbfft.RaggedPlan(sizes, offs) as p:
        d_in, d_out = run_plan(p, flat)                 # captures the graph on (d_in, d_out)
        ref = d_out.clone()
        d_in2 = d_in.clone()
        d_out2 = torch.zeros_like(d_in)
        p.execute(d_in2, d_out2)                        # patched kernel-node parameters
        p.execute(d_in2, d_in2)                         # in place, patched again
        torch.cuda.synchronize()
        assert torch.equal(d_out2, ref)
        assert torch.equal(d_in2, ref)
    check_all(to_np(ref), flat, sizes, offs)


def test_autotuned_plan_matches_oracle_and_is_deterministic():
    """The autotuner may change tile shapes, queue order, padding (none of
    which changes a single bit) and radix schedules (which change the rounding
    order): after tuning every transform still matches the oracle, and
    repeated executions of the tuned plan are bit-identical."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    sizes, offs, flat = ragged_case(3000, seed=SEED + 2)
    with gbfft.RaggedPlan(sizes, offs) as p:
        d_in, d_out = run_plan(p, flat)
        ms = p.autotune(d_in, d_out, reps=3)
        assert ms > 0
        splits = {n: gbfft.gbfft_ragged_tile_split(p.handle, n) for n in set(sizes.tolist())}
        assert set(splits.values()) <= {1, 2, 4, 8}
        for n in set(sizes.tolist()):
            rad = gbfft.gbfft_ragged_schedule(p.handle, n)
            assert rad and int(np.prod(rad)) == n
        d_out.fill_(float("nan"))
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        first = d_out.clone()
        d_out.fill_(float("nan"))
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert torch.equal(d_out, first)
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
    check_all(to_np(first), flat, sizes, offs)


def test_not_ready_item_times_out_and_is_skipped():
    """Failure injection on the host: one queue item is never published.  The
    kernel's bounded wait expires, the status word reads TIMEOUT, that item's
    rows keep the canary, every other transform is still correct, and the plan
    works again once the item is ready."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    sizes, offs, flat = ragged_case(400, seed=SEED + 3)
    with gbfft.RaggedPlan(sizes, offs) as p:
        gbfft.gbfft_ragged_set_wait_limit(p.handle, 20_000_000)  # 20 ms
        gbfft.gbfft_ragged_set_item_ready(p.handle, 0, 0)
        d_in, d_out = run_plan(p, flat)
        assert gbfft.gbfft_plan_device_status(p.handle) == gbfft.GBFFT_ERR_TIMEOUT
        y = to_np(d_out)
        untouched = [i for i, (n, o) in enumerate(zip(sizes, offs)) if np.all(np.isnan(y[o:o + n]))]
        assert 1 <= len(untouched) <= 512  # exactly the rows of one item: one length, at most one tile
        assert all(sizes[i] == sizes[untouched[0]] for i in untouched)
        check_all(y, flat, sizes, offs, skip=set(untouched))
        gbfft.gbfft_ragged_set_item_ready(p.handle, 0, 1)
        d_out.fill_(float("nan"))
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
        check_all(to_np(d_out), flat, sizes, offs)


@pytest.mark.parametrize("direction", [-1, 1])
def test_ragged_any_7_smooth_length(direction):
    """Lengths outside the power-of-two families (odd, prime powers of 3, 5, 7,
    mixed products, 1, 2 and the 8192 maximum), several transforms each,
    interleaved at odd offsets, every candidate schedule tried by the
    autotuner: every transform matches the oracle."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    lens = [1, 2, 3, 5, 6, 7, 9, 15, 21, 25, 27, 35, 45, 49, 63, 81, 105, 125, 343, 625, 729, 1000, 2401,
            3125, 6000, 6561, 8192, 7203, 4725]
    rng = np.random.Generator(np.random.Philox(key=SEED))
    sizes = np.asarray([lens[i % len(lens)] for i in range(5 * len(lens))], dtype=np.int64)
    rng.shuffle(sizes)
    gaps = rng.integers(0, 3, size=sizes.size)
    offs = np.zeros(sizes.size, dtype=np.int64)
    pos = 0
    for i, (n, g) in enumerate(zip(sizes, gaps)):
        pos += int(g)
        offs[i] = pos
        pos += int(n)
    flat = synth.uniform_flat(SEED + 7, 0, pos)
    with gbfft.RaggedPlan(sizes, offs, direction) as p:
        d_in, d_out = run_plan(p, flat)
        check_all(to_np(d_out), flat, sizes, offs, direction)
        for n in lens:
            rad = gbfft.gbfft_ragged_schedule(p.handle, n)
            assert int(np.prod(rad)) == n and all(r in (2, 3, 4, 5, 7, 8, 16) for r in rad)
        p.autotune(d_in, d_out, reps=1)
        d_out.fill_(float("nan"))
        p.execute(d_in, d_out)
        torch.cuda.synchronize()
        assert gbfft.gbfft_plan_device_status(p.handle) == 0
        check_all(to_np(d_out), flat, sizes, offs, direction)


def test_ragged_errors():
    from paper_2207_06803_gb300 import gbfft
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_ragged([8, 11], [0, 8])
    assert e.value.status == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
    for bad in (8 * 11, 13, 16384, 0):
        with pytest.raises(gbfft.GbfftError):
            gbfft.gbfft_plan_ragged([bad], [0])
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_ragged([16, 16], [0, 8])
    assert e.value.status == gbfft.GBFFT_ERR_OVERLAP
    with pytest.raises(gbfft.GbfftError) as e:
        gbfft.gbfft_plan_ragged([16], [-1])
    assert e.value.status == gbfft.GBFFT_ERR_INVALID_ARG
    with gbfft.RaggedPlan([16, 8192, 9], [0, 16, 8208]) as p:
        assert gbfft.gbfft_ragged_engine(p.handle, 9) == 0      # no compiled schedule for 9
        assert gbfft.gbfft_ragged_engine(p.handle, 32) == -1    # not in the plan
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_ragged_set_engine(p.handle, 9, 1)
        assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND
        with pytest.raises(gbfft.GbfftError):
            gbfft.gbfft_execute(p.handle, 0, 0)
        with pytest.raises(gbfft.GbfftError) as e:
            gbfft.gbfft_ragged_set_item_ready(p.handle, 99, 1)
        assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND
