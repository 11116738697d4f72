"""Tensor-core class on the GPU (radix-16 stages as DFT matmuls, FP32
accumulation) against the FP64 oracle: the tcgen05 kernel (variant 0, every
length 2^4 .. 2^14) and the warp-level MMA kernel (variant 1, 16 / 256 / 4096).

Tolerances (relative L2 per transform): FP16 2e-3; split BF16x3 5e-6 log2 N;
plain BF16 5e-3.  Plain BF16 keeps 8 significant bits: rounding both the stage
inputs and the DFT matrix gives about 3.5e-3 at N = 4096 (three stages), above
the 2e-3 aimed for; the bound here is what that arithmetic reaches, and the
miss is recorded in the design notes."""
import json

import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {1: lambda n: 2e-3, 2: lambda n: 5e-3, 3: lambda n: 5e-6 * np.log2(n)}
NAMES = {0: "fp32", 1: "tc_fp16", 2: "tc_bf16", 3: "tc_bf16x3"}


def _run(gb, x_np, n, direction, precision, variant=0):
    x = torch.from_numpy(x_np).cuda()
    with gb.Plan(n, x_np.shape[0], direction, precision, variant=variant) as p:
        y = p.execute(x)
        gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)
    return y.cpu().numpy()


@pytest.mark.parametrize("logn", range(4, 15))
@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("direction", [-1, 1])
def test_tcgen05_class(gb, oracle, logn, precision, direction):
    """The tcgen05 kernel (radix-16 UMMA stages after a radix-2/4/8 FP32
    first stage where N is not a power of 16) at every length it covers: five
    full tiles and a ragged one."""
    n = 2 ** logn
    batch = max(4096 // n, 1) * 5 + 3
    x = synth.uniform(9500 + n + precision, batch, n)
    y = _run(gb, x, n, direction, precision)
    err = oracle.rel_l2(y, oracle.fft(x, direction))
    assert np.max(err) <= TOL[precision](n), float(np.max(err))


@pytest.mark.parametrize("n", [16, 256, 4096])
@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("direction", [-1, 1])
def test_warp_mma_class(gb, oracle, n, precision, direction):
    """The warp-level MMA form (variant 1) of the same class."""
    batch = 4096 // n * 5 + 3
    x = synth.uniform(9500 + n + precision, batch, n)
    y = _run(gb, x, n, direction, precision, variant=1)
    err = oracle.rel_l2(y, oracle.fft(x, direction))
    assert np.max(err) <= TOL[precision](n), float(np.max(err))


@pytest.mark.parametrize("logn", [12, 13, 14])
@pytest.mark.parametrize("precision", [2, 3])
def test_tcgen05_many_tiles_per_cta(gb, oracle, logn, precision):
    """A batch of many tiles per CTA of the persistent grid (the tensor memory,
    mbarrier phases and DFT matrix carried from tile to tile), sampled."""
    n = 2 ** logn
    batch = (1 << 24) // n + 1
    x_np = synth.uniform(9700 + logn + precision, batch, n)
    x = torch.from_numpy(x_np).cuda()
    with gb.Plan(n, batch, -1, precision) as p:
        y = p.execute(x)
        gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)
    idx = np.unique(np.concatenate([[0, batch - 1], np.arange(1, batch, 997)]))
    ys = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    err = oracle.rel_l2(ys, oracle.fft_select(x_np, idx, -1))
    assert np.max(err) <= TOL[precision](n), float(np.max(err))


# Six-step plans round the data at the tensor-core stages of both passes (up
# to six): plain BF16, at about 2e-3 per rounded stage in quadrature, is held
# to 7e-3 there; the other classes keep their single-pass bounds.
SIX_STEP_TOL = {1: lambda n: 2e-3, 2: lambda n: 7e-3, 3: lambda n: 5e-6 * np.log2(n)}


@pytest.mark.parametrize("logn,batch", [(15, 3), (16, 2), (19, 2), (20, 1), (22, 1), (24, 1)])
@pytest.mark.parametrize("precision", [1, 2, 3])
def test_tcgen05_six_step(gb, oracle, logn, batch, precision):
    """Lengths above 2^14 in the tensor-core classes: transpose, tensor-core
    rows of N1, transpose with the six-step twiddle, rows of N2, transpose."""
    n = 2 ** logn
    x = synth.uniform(9800 + logn + precision, batch, n)
    d = -1 if logn % 2 else 1
    y = _run(gb, x, n, d, precision)
    err = oracle.rel_l2(y, oracle.fft(x, d))
    assert np.max(err) <= SIX_STEP_TOL[precision](n), float(np.max(err))


def test_tcgen05_six_step_in_place_and_sub_batches(gb, oracle):
    """in == out, and a batch above 2^28 / N (two sub-batches sharing the
    workspace), sampled against the oracle."""
    n = 2 ** 15
    batch = 2 ** 28 // n + 3
    x_np = synth.uniform(9850, batch, n)
    x = torch.from_numpy(x_np).cuda()
    with gb.Plan(n, batch, -1, 3) as p:
        assert p.describe()["chunk_batch"] == 2 ** 28 // n
        p.execute(x, x)
        gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)
    idx = np.array([0, 1, batch // 2, 2 ** 28 // n - 1, 2 ** 28 // n, batch - 1])
    ys = x[torch.from_numpy(idx).cuda()].cpu().numpy()
    err = oracle.rel_l2(ys, oracle.fft_select(x_np, idx, -1))
    assert np.max(err) <= SIX_STEP_TOL[3](n), float(np.max(err))


def test_tcgen05_six_step_host_graph_and_server(gb, oracle):
    """A six-step tensor-core plan through fft_execute_host (pinned host
    buffers, chunked copies), through fft_execute_graph, and as a server job:
    the same bytes as fft_execute."""
    n, batch, prec = 2 ** 16, 5, 1
    x_np = synth.uniform(9860, batch, n)
    x = torch.from_numpy(x_np).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    with gb.Plan(n, batch, 1, prec) as p:
        ref = p.execute(x)
        g = p.execute_graph(x)
        hin = torch.from_numpy(x_np).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        din, dout = torch.empty_like(x), torch.empty_like(x)
        p.execute_host(hin, hout, din, dout)
        torch.cuda.synchronize()
        gb.fft_plan_sync_status(p.handle, stream)
    assert torch.equal(ref, g)
    assert torch.equal(ref.cpu(), hout)
    out = torch.empty_like(x)
    torch.cuda.synchronize()
    srv = gb.fft_server_create(memory_budget_bytes=1 << 30, streams=2)
    try:
        t = gb.fft_server_submit(srv, n, batch, 1, prec, x.data_ptr(), out.data_ptr())
        assert gb.fft_server_wait(srv, t, 60.0)["status"] == 0
    finally:
        gb.fft_server_destroy(srv)
    torch.cuda.synchronize()
    assert torch.equal(ref, out)
    err = oracle.rel_l2(ref.cpu().numpy(), oracle.fft(x_np, 1))
    assert np.max(err) <= SIX_STEP_TOL[prec](n), float(np.max(err))


def test_tc_rejects_other_lengths(gb):
    for n, variant in ((2 ** 25, 0), (8, 0), (1024, 1)):
        with pytest.raises(gb.GbfftError) as e:
            gb.fft_plan_create(n, 4, -1, 2, variant=variant)
        assert e.value.status == gb.FFT_ERR_NOT_IMPLEMENTED, (n, variant)


def test_tc_buried_tone_accuracy_report(gb, oracle, capsys):
    """N = 4096, batch 32768: uniform noise plus a 1e-3 tone per transform.
    Relative L2 per precision class and the error at the tone's bin relative
    to the tone's exact contribution N * 1e-3 (sampled transforms)."""
    n, batch = 4096, 32768
    x, bins = synth.buried_tone(8000, batch, n)
    xt = torch.from_numpy(x).cuda()
    idx = np.arange(0, batch, 1023)
    ref = oracle.fft_select(x, idx)
    report = {}
    for prec, variant in ((0, 0), (1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)):
        with gb.Plan(n, batch, -1, prec, variant=variant) as p:
            y = p.execute(xt)
            torch.cuda.synchronize()
        ys = y[torch.from_numpy(idx).cuda()].cpu().numpy()
        err = oracle.rel_l2(ys, ref)
        tone = np.abs(ys[np.arange(idx.size), bins[idx]] - ref[np.arange(idx.size), bins[idx]])
        name = NAMES[prec] + ("_warp_mma" if variant == 1 else "")
        report[name] = {"rel_l2_max": float(err.max()), "rel_l2_mean": float(err.mean()),
                        "tone_bin_err_rel": float(tone.max() / (n * 1e-3))}
        tol = 1e-6 * np.log2(n) if prec == 0 else TOL[prec](n)
        assert err.max() <= tol
    with capsys.disabled():
        print("TC_ACCURACY " + json.dumps(report))


@pytest.mark.parametrize("n", [16, 256, 4096])
@pytest.mark.parametrize("precision", [1, 3])
@pytest.mark.parametrize("variant", [0, 1])
def test_tc_staged_and_unaligned_input(gb, oracle, n, precision, variant):
    """The kernel copies each next tile into shared memory when the input is
    16-byte aligned and reads global memory directly when it is only 8-byte
    aligned; both give the same accuracy (a ragged last tile, many tiles per
    block of the persistent grid), and on tcgen05 the same bytes."""
    batch = (4096 // n) * 700 + 5
    x_np = synth.uniform(9600 + n + precision, batch, n)
    buf = torch.zeros(batch * n + 1, dtype=torch.complex64, device="cuda")
    ref = oracle.fft(x_np, -1)
    outs = []
    for shift in (0, 1):
        xin = buf[shift:shift + batch * n]
        xin.copy_(torch.from_numpy(x_np.reshape(-1)))
        out = torch.empty(batch * n, dtype=torch.complex64, device="cuda")
        with gb.Plan(n, batch, -1, precision, variant=variant) as p:
            st = torch.cuda.current_stream().cuda_stream
            gb.fft_execute(p.handle, xin.data_ptr(), out.data_ptr(), st)
            gb.fft_plan_sync_status(p.handle, st)
        err = oracle.rel_l2(out.view(batch, n).cpu().numpy(), ref)
        assert np.max(err) <= TOL[precision](n), (shift, float(np.max(err)))
        outs.append(out)
    if variant == 0:
        assert torch.equal(outs[0], outs[1])
