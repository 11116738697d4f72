"""Serving policy (csrc/scheduler.h) on a simulated device, CPU only:
admission never exceeds the memory budget, in strict arrival order the oldest
waiting job always goes first, only same-key jobs share a launch, jobs that
arrive while others run are admitted as memory frees up, jobs larger than the
budget are rejected, and backfilled jobs never delay the waiting head when
the run-time estimates are exact."""
import numpy as np

from serve import sched


def _random_stream(seed, n=400):
    rng = np.random.default_rng(seed)
    key = rng.integers(0, 6, n)
    nbytes = (2 ** rng.integers(20, 30, n)).astype(np.uint64)
    arrive = np.sort(rng.integers(0, 300, n))
    dur = rng.integers(1, 20, n)
    grp = rng.integers(0, 2, n)
    return key, nbytes, arrive, dur, grp


def test_budget_and_completion():
    key, nbytes, arrive, dur, grp = _random_stream(1)
    budget = 4 << 30
    r = sched.simulate(key, nbytes, arrive, dur, grp, budget)
    assert r["steps"] > 0                       # -1 would mean the budget was exceeded
    assert r["peak"] <= budget
    assert not r["rejected"].any()
    assert (r["done"] >= 0).all() and (r["launch"] >= arrive).all()


def test_groups_share_one_key_and_are_groupable():
    key, nbytes, arrive, dur, grp = _random_stream(2)
    r = sched.simulate(key, nbytes, arrive, dur, grp, 8 << 30)
    for g in np.unique(r["group"]):
        members = np.where(r["group"] == g)[0]
        assert len(set(key[members])) == 1
        if len(members) > 1:
            assert grp[members].all()
    assert len(np.unique(r["group"])) < len(key)      # some coalescing happened


def test_oldest_first():
    """Every launch contains the oldest job still waiting: groups launch in the
    order of their oldest member (later same-key jobs may join it early, which
    never delays an older job)."""
    key, nbytes, arrive, dur, grp = _random_stream(3)
    r = sched.simulate(key, nbytes, arrive, dur, grp, 2 << 30)
    groups = {}
    for j, g in enumerate(r["group"]):
        groups.setdefault(g, []).append(j)
    firsts = sorted((r["launch"][m[0]], g, min(m)) for g, m in groups.items())
    oldest = [f[2] for f in firsts]            # job indices are in arrival order
    assert oldest == sorted(oldest)


def test_continuous_admission():
    """Memory held by one long job: later small jobs run as soon as their bytes
    fit, while the long job is still running."""
    key = [0, 1, 1, 1]
    nbytes = [6 << 30, 1 << 30, 1 << 30, 1 << 30]
    arrive = [0, 1, 2, 3]
    dur = [100, 5, 5, 5]
    r = sched.simulate(key, nbytes, arrive, dur, [0, 1, 1, 1], 8 << 30)
    assert r["launch"][0] == 0
    assert (r["launch"][1:] < 100).all()             # admitted while job 0 runs
    assert r["peak"] <= 8 << 30


def test_too_large_is_rejected():
    r = sched.simulate([0, 0], [16 << 30, 1 << 20], [0, 0], [1, 1], [1, 1], 8 << 30)
    assert r["rejected"].tolist() == [True, False]
    assert r["done"][1] >= 0


def test_backfill_never_delays_the_head():
    """Backfilling with exact run-time estimates.  Job 0 (5 GB, 100 steps) runs;
    job 1 (7 GB) waits for it: its reservation is step 100 with 3 GB left over
    next to it.  Job 2 (4 GB, 200 steps) fits now but would still hold 4 GB at
    step 100, more than the 3 GB left over: it waits.  Job 3 (4 GB, 50 steps)
    ends before step 100: it starts at once.  Job 4 (2 GB, 500 steps) fits in
    the 3 GB next to job 1: it starts as soon as job 3's bytes free up.  Job 1
    still starts at step 100, exactly as in strict arrival order."""
    G = 1 << 30
    key = [0, 1, 2, 3, 4]
    nbytes = [5 * G, 7 * G, 4 * G, 4 * G, 2 * G]
    arrive = [0, 1, 2, 3, 4]
    dur = [100, 10, 200, 50, 500]
    grp = [0] * 5
    fifo = sched.simulate(key, nbytes, arrive, dur, grp, 10 * G, backfill=False)
    bf = sched.simulate(key, nbytes, arrive, dur, grp, 10 * G, backfill=True)
    assert fifo["launch"].tolist() == [0, 100, 110, 110, 110]
    assert bf["launch"].tolist() == [0, 100, 110, 3, 53]
    assert bf["peak"] <= 10 * G and fifo["peak"] <= 10 * G


def test_backfill_random_streams():
    """Random streams under a tight budget: with backfilling every job still
    completes, the budget holds, only same-key jobs share a launch, and the
    mean wait for a launch is no longer than in strict arrival order."""
    for seed in (11, 12, 13, 14):
        key, nbytes, arrive, dur, grp = _random_stream(seed)
        budget = 2 << 30
        fifo = sched.simulate(key, nbytes, arrive, dur, grp, budget, backfill=False)
        bf = sched.simulate(key, nbytes, arrive, dur, grp, budget, backfill=True)
        assert bf["steps"] > 0 and bf["peak"] <= budget
        assert (bf["done"] >= 0).all() and (bf["launch"] >= arrive).all()
        for g in np.unique(bf["group"]):
            members = np.where(bf["group"] == g)[0]
            assert len(set(key[members])) == 1
        assert np.mean(bf["launch"] - arrive) <= np.mean(fifo["launch"] - arrive)


def test_backfilled_group_coalesces_same_key_jobs():
    """A blocked head does not stop later same-key small jobs from starting
    together in one backfilled group, and the group as a whole obeys the
    reservation: job 1 (7 GB) waits for job 0 (5 GB, 100 steps); jobs 2-4
    (1 GB, 10 steps each, same key, groupable) run back to back in one group
    that ends at step 32 < 100; the head still starts at step 100."""
    G = 1 << 30
    key = [0, 1, 2, 2, 2]
    nbytes = [5 * G, 7 * G, G, G, G]
    arrive = [0, 1, 2, 2, 2]
    dur = [100, 10, 10, 10, 10]
    grp = [0, 0, 1, 1, 1]
    r = sched.simulate(key, nbytes, arrive, dur, grp, 10 * G, backfill=True)
    assert r["launch"].tolist() == [0, 100, 2, 2, 2]
    assert len(set(r["group"][2:].tolist())) == 1          # one coalesced group
    assert r["done"][2] == 32 and r["peak"] <= 10 * G
