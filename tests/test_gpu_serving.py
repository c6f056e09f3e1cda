"""Serving loop: continuous batching under a device-memory budget.  Each
result in a concurrent mix equals the same request run alone (bit for bit:
a row's arithmetic does not depend on what it is batched with) and the FP64
oracle within tolerance; admission respects the budget; latency statistics
are consistent."""
import numpy as np
import pytest

import oracle
from helpers import ncpu, row_rel_l2, tol_fp32
from paper_2207_06803_gb300 import synth

pytestmark = pytest.mark.gpu
SEED = synth.DEFAULT_SEED


def make_requests(count, seed, max_batch=32, lo=16, hi=16384):
    import torch
    fam = np.asarray(synth.size_family(lo, hi))
    rng = np.random.Generator(np.random.Philox(key=seed))
    ns = fam[rng.integers(0, fam.size, size=count)]
    bs = rng.integers(1, max_batch + 1, size=count)
    dirs = np.where(rng.random(count) < 0.5, -1, 1)
    ins, outs = [], []
    for i in range(count):
        x = synth.uniform_flat(seed + i, 0, int(ns[i] * bs[i]))
        ins.append(torch.from_numpy(x.view(np.float32)).pin_memory())
        outs.append(torch.full_like(ins[-1], float("nan")).pin_memory())
    return ns, bs, dirs, ins, outs


def test_mix_equals_alone_and_oracle():
    import torch
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(160, SEED)
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=4) as srv:
        arrivals = np.sort(np.random.default_rng(1).uniform(0, 0.02, size=len(ns)))
        tickets = srv.replay(ns, bs, dirs, ins, outs, arrivals)
        for t in tickets:
            srv.wait(t, 60.0)
            done, lat = srv.poll(t)
            assert done == 1 and lat > 0
            queued, lat2 = srv.timing(t)
            assert lat2 == lat and 0 <= queued <= lat
        st = srv.stats()
        assert st["completed"] == len(ns)
        assert 0 < st["p50_s"] <= st["p99_s"] <= st["max_s"]
        assert st["groups"] <= len(ns) and st["max_arena_bytes"] <= (256 << 20)
    # each request alone, through the same kind of server with nothing else in flight (a request's rows
    # are cut into the same queue items whatever else shares the launch)
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=1) as alone:
        for i in range(len(ns)):
            solo = torch.full_like(ins[i], float("nan")).pin_memory()
            alone.wait(alone.submit(int(ns[i]), int(bs[i]), int(dirs[i]), ins[i], solo), 60.0)
            assert torch.equal(solo, outs[i]), i
    for i in range(0, len(ns), 7):
        n, b = int(ns[i]), int(bs[i])
        x = ins[i].numpy().view(np.complex64).reshape(b, n)
        y = outs[i].numpy().view(np.complex64).reshape(b, n)
        ref = oracle.dft(x.astype(np.complex128), int(dirs[i]), nthreads=ncpu())
        assert row_rel_l2(y, ref).max() <= tol_fp32(n), (i, n)


def test_small_budget_queues_and_completes():
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(60, SEED + 5, max_batch=64, lo=1024, hi=16384)
    budget = 24 << 20
    with gbfft.Server(mem_budget_bytes=budget, n_streams=3) as srv:
        tickets = [srv.submit(int(n), int(b), int(d), i, o) for n, b, d, i, o in zip(ns, bs, dirs, ins, outs)
                   if 16 * n * b + 512 <= budget]
        for t in tickets:
            srv.wait(t, 60.0)
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["max_arena_bytes"] <= budget


def test_budget_and_argument_errors():
    import torch
    from paper_2207_06803_gb300 import gbfft
    with gbfft.Server(mem_budget_bytes=4 << 20, n_streams=2) as srv:
        big = torch.zeros(2 * 16384 * 64).pin_memory()
        with pytest.raises(gbfft.GbfftError) as e:
            srv.submit(16384, 64, -1, big, big)  # 8 MiB slot > 4 MiB budget
        assert e.value.status == gbfft.GBFFT_ERR_BUDGET
        small = torch.zeros(2 * 11 * 2).pin_memory()
        with pytest.raises(gbfft.GbfftError) as e:
            srv.submit(11, 2, -1, small, small)
        assert e.value.status == gbfft.GBFFT_ERR_UNSUPPORTED_SIZE
        with pytest.raises(gbfft.GbfftError) as e:
            srv.poll(12345)
        assert e.value.status == gbfft.GBFFT_ERR_NOT_FOUND


def test_destroy_with_work_outstanding_does_not_hang():
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(40, SEED + 9, max_batch=128, lo=4096, hi=16384)
    srv = gbfft.Server(mem_budget_bytes=16 << 20, n_streams=2)
    for n, b, d, i, o in zip(ns, bs, dirs, ins, outs):
        if 16 * n * b + 512 <= (16 << 20):
            srv.submit(int(n), int(b), int(d), i, o)
    srv.close()  # cancels what is queued, waits for what runs


def test_serial_and_per_length_servers_agree_with_the_oracle():
    """The naive queue (one request at a time) and per-length batching run the
    single-pass / two-pass kernels instead of the ragged launch: bit for bit
    the same as each other, and within tolerance of the oracle."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(40, SEED + 3)
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=3, per_length=True) as srv:
        for t in srv.replay(ns, bs, dirs, ins, outs, np.linspace(0, 0.01, len(ns))):
            srv.wait(t, 60.0)
        assert srv.stats()["completed"] == len(ns)
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=1, serial=True) as alone:
        for i in range(len(ns)):
            solo = torch.full_like(ins[i], float("nan")).pin_memory()
            alone.wait(alone.submit(int(ns[i]), int(bs[i]), int(dirs[i]), ins[i], solo), 60.0)
            assert torch.equal(solo, outs[i]), i
    for i in range(0, len(ns), 3):
        n, b = int(ns[i]), int(bs[i])
        x = ins[i].numpy().view(np.complex64).reshape(b, n)
        ref = oracle.dft(x.astype(np.complex128), int(dirs[i]), nthreads=ncpu())
        assert row_rel_l2(outs[i].numpy().view(np.complex64).reshape(b, n), ref).max() <= tol_fp32(n), (i, n)


def test_device_buffers_and_phases():
    """Requests whose input and output live in device memory, on a server
    that times every group's phases: the results match host-buffer requests
    bit for bit, and each request's phases add up to its latency."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(48, SEED + 4)
    d_ins = [t.cuda() for t in ins]
    d_outs = [torch.full_like(t, float("nan")) for t in d_ins]
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=4, phases=True) as srv:
        tickets = srv.replay(ns, bs, dirs, d_ins, d_outs, np.linspace(0, 0.01, len(ns)))
        for t in tickets:
            srv.wait(t, 60.0)
        for t in tickets:
            ph = srv.phases(t)
            assert all(np.isfinite(v) for v in ph.values())
            assert ph["h2d_s"] >= 0 and ph["kernel_s"] >= 0 and ph["d2h_s"] >= 0 and ph["queued_s"] >= 0
            parts = sum(v for k, v in ph.items() if k != "latency_s")
            assert abs(parts - ph["latency_s"]) <= 1e-6 + 1e-9 * ph["latency_s"]
        for t in tickets:
            srv.release(t)
        for t in srv.replay(ns, bs, dirs, ins, outs, np.linspace(0, 0.01, len(ns))):
            srv.wait(t, 60.0)
    torch.cuda.synchronize()
    for i in range(len(ns)):
        assert torch.equal(d_outs[i].cpu(), outs[i]), i


def test_direct_and_staged_ragged_launches_agree():
    """Pinned host buffers are read and written by the ragged launch directly
    (over the host link) or copied through the device arena (staged): the
    same kernel on the same queue items, so the results agree bit for bit."""
    import torch
    from paper_2207_06803_gb300 import gbfft
    ns, bs, dirs, ins, outs = make_requests(64, SEED + 6, hi=8192)
    staged_out = [torch.full_like(t, float("nan")).pin_memory() for t in ins]
    arrivals = np.linspace(0, 0.01, len(ns))
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=4) as srv:
        for t in srv.replay(ns, bs, dirs, ins, outs, arrivals):
            srv.wait(t, 60.0)
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=4, staged=True) as srv:
        for t in srv.replay(ns, bs, dirs, ins, staged_out, arrivals):
            srv.wait(t, 60.0)
    for i in range(len(ns)):
        assert torch.equal(staged_out[i], outs[i]), i
