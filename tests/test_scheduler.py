"""Serving policy (csrc/scheduler.h) on a simulated device, CPU only:
admission never exceeds the memory budget, the oldest waiting job always goes
first, only same-key jobs share a launch, jobs that arrive while others run
are admitted as memory frees up, and jobs larger than the budget are
rejected."""
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
