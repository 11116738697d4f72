"""The work queue's host bookkeeping (csrc/queue_ring.h) against a model of
its ring, on the CPU: a worker completing tickets in order at random moments
and a host submitting and scanning for completions at random moments, with
slots reused and completed again between scans.  The equality form of the
scan (a ticket counted complete only while its slot still shows it) is
replayed too, to show that these interleavings catch it."""
import pytest

from emu import emu


@pytest.mark.parametrize("slots", [1, 2, 4, 7, 64])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ring_bookkeeping(slots, seed):
    assert emu.ring_replay(seed, slots, 20000) == ""


@pytest.mark.parametrize("slots", [2, 4])
def test_equality_scan_loses_completions(slots):
    failures = [emu.ring_replay(seed, slots, 20000, exact=True) for seed in range(1, 6)]
    assert any(f for f in failures), failures
