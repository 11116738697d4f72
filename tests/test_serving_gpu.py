"""Serving loop on the GPU: a mixed stream of jobs (shapes, batches,
directions, precisions) submitted while others run; every job's output equals
the same job run alone through its own plan (within the tolerance of its
precision class) and a sample matches the FP64 oracle; the memory budget holds;
host-side faults surface as job errors."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: lambda n: 1e-6 * max(1.0, np.log2(n)), 1: lambda n: 2e-3, 2: lambda n: 5e-3,
       3: lambda n: 5e-6 * np.log2(n)}


def _mix(seed, count):
    rng = np.random.default_rng(seed)
    shapes = [(256,), (1024,), (4096,), (2 ** 14,), (2 ** 16,), (2 ** 20,), (64, 128)]
    jobs = []
    for i in range(count):
        shape = shapes[rng.integers(len(shapes))]
        n = int(np.prod(shape))
        prec = 0
        if len(shape) == 1 and n <= 2 ** 14 and rng.random() < 0.4:  # tensor-core class
            prec = int(rng.integers(1, 4))
        batch = int(rng.integers(1, max(2, min(64, 2 ** 22 // n))))
        d = -1 if rng.random() < 0.5 else 1
        jobs.append((shape, batch, d, prec))
    return jobs


def test_mixed_stream_matches_alone(gb, oracle):
    jobs = _mix(11, 48)
    bufs, tickets = [], []
    for k, (shape, batch, d, prec) in enumerate(jobs):
        n = int(np.prod(shape))
        x = torch.from_numpy(synth.uniform(12000 + k, batch, n)).cuda()
        bufs.append((x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    srv = gb.fft_server_create(memory_budget_bytes=512 << 20, streams=4)
    try:
        # the first half arrives as one held burst (coalesced), the second half
        # one by one while the first half runs
        gb.fft_server_pause(srv, True)
        for k, ((shape, batch, d, prec), (x, y)) in enumerate(zip(jobs, bufs)):
            if k == len(jobs) // 2:
                gb.fft_server_pause(srv, False)
            tickets.append(gb.fft_server_submit(srv, shape if len(shape) > 1 else shape[0], batch,
                                                d, prec, x.data_ptr(), y.data_ptr()))
        results = [gb.fft_server_wait(srv, t, 120.0) for t in tickets]
        stats = gb.fft_server_stats(srv)
    finally:
        gb.fft_server_destroy(srv)
    assert all(r["status"] == 0 for r in results)
    assert stats["completed"] == len(jobs) and stats["failed"] == 0
    assert stats["peak_bytes_in_flight"] <= 512 << 20
    assert stats["groups"] < len(jobs) and stats["coalesced_jobs"] > 0   # coalescing happened
    assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    torch.cuda.synchronize()
    for k, ((shape, batch, d, prec), (x, y)) in enumerate(zip(jobs, bufs)):
        n = int(np.prod(shape))
        with gb.Plan(shape if len(shape) > 1 else shape[0], batch, d, prec) as p:
            alone = p.execute(x)
            torch.cuda.synchronize()
        ym, ya = y.cpu().numpy().reshape(batch, -1), alone.cpu().numpy().reshape(batch, -1)
        assert np.max(oracle.rel_l2(ym, ya)) <= TOL[prec](n), (k, shape, batch, prec)
        if k % 6 == 0:                                     # sample against the oracle
            xn = x.cpu().numpy().reshape((batch,) + shape)
            ref = oracle.fft(xn, d) if len(shape) == 1 else oracle.fft2d(xn, d)
            assert np.max(oracle.rel_l2(ym, ref.reshape(batch, -1))) <= TOL[prec](n)


def test_budget_rejection_and_fault_injection(gb):
    srv = gb.fft_server_create(memory_budget_bytes=64 << 20, fail_workspace_alloc=1)
    try:
        big = torch.zeros(2 ** 22, dtype=torch.complex64, device="cuda")
        with pytest.raises(gb.GbfftError) as e:      # 2 x 32 MiB + workspace > 64 MiB
            gb.fft_server_submit(srv, 2 ** 22, 1, -1, 0, big.data_ptr(), big.data_ptr())
        assert e.value.status == gb.FFT_ERR_OUT_OF_MEMORY
        x = torch.ones(2 ** 16, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(x)
        t_multi = gb.fft_server_submit(srv, 2 ** 16, 1, -1, 0, x.data_ptr(), y.data_ptr())
        xs = torch.ones(4096, dtype=torch.complex64, device="cuda")
        ys = torch.empty_like(xs)
        t_single = gb.fft_server_submit(srv, 1024, 4, -1, 0, xs.data_ptr(), ys.data_ptr())
        r_multi = gb.fft_server_wait(srv, t_multi, 60.0)
        r_single = gb.fft_server_wait(srv, t_single, 60.0)
        assert r_multi["status"] == gb.FFT_ERR_OUT_OF_MEMORY   # workspace allocation refused
        assert r_single["status"] == 0                        # one-pass job needs no workspace
        torch.cuda.synchronize()
        assert torch.allclose(ys.view(4, 1024)[:, 0], torch.full((4,), 1024.0 + 0j, device="cuda",
                                                                   dtype=torch.complex64))
        with pytest.raises(gb.GbfftError):
            gb.fft_server_submit(srv, 12, 1, -1, 0, x.data_ptr(), y.data_ptr())
    finally:
        gb.fft_server_destroy(srv)


@pytest.mark.parametrize("strict", [0, 1])
def test_backfill_small_job_passes_a_blocked_head(gb, oracle, strict):
    """Two two-pass jobs that do not fit the budget together and a small job
    behind them, admitted as one held burst: the second large job waits for
    the first one's memory.  With backfilling the small job starts at once
    (its estimated run time ends long before the first job frees its bytes);
    in strict arrival order nothing is admitted out of order.  Every result
    matches the same job run alone."""
    specs = [(2 ** 20, 16), (2 ** 20, 16), (1024, 8)]
    bufs = []
    for k, (n, b) in enumerate(specs):
        x = torch.from_numpy(synth.uniform(13000 + k, b, n)).cuda()
        bufs.append((x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    srv = gb.fft_server_create(memory_budget_bytes=600 << 20, streams=4, strict_order=strict)
    try:
        gb.fft_server_pause(srv, True)
        tickets = [gb.fft_server_submit(srv, n, b, -1, 0, x.data_ptr(), y.data_ptr())
                   for (n, b), (x, y) in zip(specs, bufs)]
        gb.fft_server_pause(srv, False)
        results = [gb.fft_server_wait(srv, t, 60.0) for t in tickets]
        stats = gb.fft_server_stats(srv)
    finally:
        gb.fft_server_destroy(srv)
    assert all(r["status"] == 0 for r in results)
    assert stats["peak_bytes_in_flight"] <= 600 << 20
    if strict:
        assert stats["backfilled_jobs"] == 0
    else:
        # the small job launched before the second large one (which waited for
        # the first one's memory) although it was submitted after it
        assert stats["backfilled_jobs"] >= 1
        assert results[2]["queue_ms"] < results[1]["queue_ms"]
    torch.cuda.synchronize()
    for (n, b), (x, y) in zip(specs, bufs):
        with gb.Plan(n, b, -1) as p:
            alone = p.execute(x)
            torch.cuda.synchronize()
        assert np.max(oracle.rel_l2(y.cpu().numpy().reshape(b, n),
                                    alone.cpu().numpy().reshape(b, n))) <= TOL[0](n)
