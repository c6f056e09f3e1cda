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
    # each request alone, through a server that runs one request at a time
    with gbfft.Server(mem_budget_bytes=256 << 20, n_streams=1, serial=True) as alone:
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
