"""Persistent work queue (fft_queue_*): jobs run by the resident worker
against the FP64 oracle at the FP32 tolerance (1e-6 log2 N), the ring reused
many times over, in-place jobs, the worker ending when idle and started again,
and argument checks.

The worker runs on the queue's own stream, so each test makes the inputs
ready (synchronises the stream that wrote them) before submitting."""
import time

import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(n):
    return 1e-6 * np.log2(n)


def _ready():
    torch.cuda.current_stream().synchronize()


@pytest.mark.parametrize("n", [2, 16, 256, 1024, 4096])
@pytest.mark.parametrize("direction", [-1, 1])
def test_queue_jobs_match_oracle(gb, oracle, n, direction):
    """Jobs of several batch sizes (one, the largest, ragged tiles) through a
    ring of four slots (the fifth job waits for the first slot)."""
    max_batch = max(1, 65536 // n)
    batches = [1, max_batch, 3, max_batch // 2 + 1, 7]
    x_np = synth.uniform(9990 + n, sum(batches), n)
    x = torch.from_numpy(x_np).cuda()
    y = torch.zeros_like(x)
    _ready()
    with gb.Queue(n, max_batch, direction, slots=4) as q:
        tickets, off = [], 0
        for b in batches:
            tickets.append(q.submit(x[off:off + b], y[off:off + b], b))
            off += b
        for t in tickets:
            q.wait(t, 10.0)
        assert q.info()["completed"] == len(batches)
    err = oracle.rel_l2(y.cpu().numpy(), oracle.fft(x_np, direction))
    assert np.max(err) <= _tol(n), float(np.max(err))


def test_queue_ring_reused_many_times(gb, oracle):
    """100 jobs through 8 slots, submitted back to back; every job with the
    same input gives the same bytes."""
    n, B = 1024, 64
    x_np = synth.uniform(9991, 4 * B, n)
    x = torch.from_numpy(x_np).cuda()
    outs = torch.zeros(100, B, n, dtype=torch.complex64, device="cuda")
    _ready()
    with gb.Queue(n, B, -1, slots=8) as q:
        tickets = [q.submit(x[(i % 4) * B:(i % 4 + 1) * B], outs[i], B) for i in range(100)]
        q.wait(tickets[-1], 30.0)
        for t in tickets:  # completed in ticket order
            q.wait(t, 0.0)
        assert q.info()["completed"] == 100
    got = outs.cpu().numpy()
    ref = oracle.fft(x_np, -1).reshape(4, B, n)
    for i in (0, 1, 2, 3, 37, 99):
        err = oracle.rel_l2(got[i], ref[i % 4])
        assert np.max(err) <= _tol(n), (i, float(np.max(err)))
    for i in range(4, 100):
        assert np.array_equal(got[i], got[i % 4]), i


def test_queue_in_place(gb, oracle):
    n, B = 4096, 9
    x_np = synth.uniform(9992, B, n)
    x = torch.from_numpy(x_np).cuda()
    _ready()
    with gb.Queue(n, 16, 1) as q:
        q.wait(q.submit(x, x, B), 10.0)
    err = oracle.rel_l2(x.cpu().numpy(), oracle.fft(x_np, 1))
    assert np.max(err) <= _tol(n), float(np.max(err))


def test_queue_worker_ends_when_idle_and_restarts(gb, oracle):
    """With no job for well over the idle bound the worker exits; the next
    submit launches it again and the result is the same."""
    n, B = 256, 16
    x_np = synth.uniform(9993, B, n)
    x = torch.from_numpy(x_np).cuda()
    y1, y2 = torch.zeros_like(x), torch.zeros_like(x)
    _ready()
    with gb.Queue(n, B, -1) as q:
        q.wait(q.submit(x, y1, B), 10.0)
        assert q.info()["worker_launches"] == 1
        time.sleep(1.5)
        q.wait(q.submit(x, y2, B), 10.0)
        assert q.info()["worker_launches"] == 2
    assert torch.equal(y1, y2)
    err = oracle.rel_l2(y1.cpu().numpy(), oracle.fft(x_np, -1))
    assert np.max(err) <= _tol(n), float(np.max(err))


def test_queue_submit_while_another_thread_waits(gb, oracle):
    """One thread submits 64 jobs while another waits for each in turn."""
    import threading

    n, B = 512, 32
    x_np = synth.uniform(9994, B, n)
    x = torch.from_numpy(x_np).cuda()
    outs = torch.zeros(64, B, n, dtype=torch.complex64, device="cuda")
    _ready()
    errors = []
    with gb.Queue(n, B, -1, slots=4) as q:
        tickets = []
        cv = threading.Condition()

        def waiter():
            try:
                for i in range(64):
                    with cv:
                        cv.wait_for(lambda: len(tickets) > i, timeout=30)
                        t = tickets[i]
                    q.wait(t, 30.0)
            except Exception as e:  # reported below
                errors.append(e)

        th = threading.Thread(target=waiter)
        th.start()
        for i in range(64):
            t = q.submit(x, outs[i], B)
            with cv:
                tickets.append(t)
                cv.notify_all()
        th.join(60)
        assert not th.is_alive() and not errors, errors
        assert q.info()["completed"] == 64
    ref = oracle.fft(x_np, -1)
    got = outs.cpu().numpy()
    assert np.max(oracle.rel_l2(got[63], ref)) <= _tol(n)
    for i in range(64):
        assert np.array_equal(got[i], got[0]), i


def test_queue_rejects(gb):
    x = torch.zeros(64 * 1024 + 1, dtype=torch.complex64, device="cuda")
    _ready()
    with gb.Queue(1024, 64) as q:
        with pytest.raises(gb.GbfftError):
            q.submit_ptr(x.data_ptr(), x.data_ptr(), 65)      # above max_batch
        with pytest.raises(gb.GbfftError):
            q.submit_ptr(x.data_ptr(), x.data_ptr(), 0)
        with pytest.raises(gb.GbfftError):
            q.submit_ptr(x.data_ptr() + 4, x.data_ptr(), 1)   # not 8-byte aligned
        with pytest.raises(gb.GbfftError):
            q.wait(1)                                         # never issued
        assert q.info() == {"worker_launches": 0, "completed": 0}
    for n in (8192, 1000):
        with pytest.raises(gb.GbfftError):
            gb.Queue(n, 4)
