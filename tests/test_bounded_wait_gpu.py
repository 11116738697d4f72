"""Device-side failure detection without a fault: the kernels' bounded
mbarrier wait, run on a barrier that nothing completes (fft_wait_selftest),
gives up after its poll limit, reports it through a status word the host
reads, and leaves the device usable: a plan executed afterwards still matches
the FP64 oracle."""
import time

import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_device_stays_usable(gb, oracle):
    for polls in (1, 64, 4096, 1 << 16):
        t0 = time.perf_counter()
        assert gb.fft_wait_selftest(polls) == 1
        assert time.perf_counter() - t0 < 5.0
    for polls in (0, 2 ** 22 + 1):
        with pytest.raises(gb.GbfftError):
            gb.fft_wait_selftest(polls)
    # staged kernels (2^13) and a two-pass plan run normally afterwards
    for n, batch in ((8192, 33), (2 ** 20, 2)):
        x_np = synth.uniform(7100 + batch, batch, n)
        x = torch.from_numpy(x_np).cuda()
        with gb.Plan(n, batch) as p:
            y = p.execute(x)
            gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)
        err = oracle.rel_l2(y.cpu().numpy(), oracle.fft(x_np))
        assert np.max(err) <= 1e-6 * np.log2(n), float(np.max(err))
