"""The C ABI without a GPU: the library loads, exports every symbol the header
declares, plans on a described device, and fails cleanly where a GPU is
needed.  CPU only."""
import ctypes
import os
import re

import pytest

from paper_1505_08067_gb300 import gbfft as g

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"GBFFT_API[^;(]*?\b(fft_\w+)\s*\(", txt, re.S))
    return names


def test_header_symbols_exported():
    lib = ctypes.CDLL(g.LIB_PATH)
    names = _declared()
    assert len(names) >= 15
    for name in sorted(names):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_no_gpu_means_error_not_fallback():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except Exception:
        pass
    with pytest.raises(g.GbfftError) as e:
        g.fft_plan_create(1024, 4)
    assert e.value.status == g.FFT_ERR_CUDA
    # the work queue: shape errors first, then no device
    for n, st in ((8192, g.FFT_ERR_NOT_IMPLEMENTED), (1000, g.FFT_ERR_UNSUPPORTED_SIZE),
                  (1024, g.FFT_ERR_CUDA)):
        with pytest.raises(g.GbfftError) as e:
            g.Queue(n, 64)
        assert e.value.status == st
    # the bounded-wait diagnostic: argument errors first, then no device
    for polls, st in ((0, g.FFT_ERR_INVALID_ARG), (2 ** 22 + 1, g.FFT_ERR_INVALID_ARG),
                      (64, g.FFT_ERR_CUDA)):
        with pytest.raises(g.GbfftError) as e:
            g.fft_wait_selftest(polls)
        assert e.value.status == st


@pytest.mark.parametrize("n,batch,status", [
    (12, 1, g.FFT_ERR_UNSUPPORTED_SIZE), (2 ** 25, 1, g.FFT_ERR_UNSUPPORTED_SIZE),
    (0, 1, g.FFT_ERR_UNSUPPORTED_SIZE), (1024, -1, g.FFT_ERR_INVALID_ARG),
    ((2 ** 15, 8), 1, g.FFT_ERR_UNSUPPORTED_SIZE), ((3, 8), 1, g.FFT_ERR_UNSUPPORTED_SIZE)])
def test_dry_run_rejects(n, batch, status):
    with pytest.raises(g.GbfftError) as e:
        g.fft_plan_dry_run(n, batch)
    assert e.value.status == status


def test_dry_run_rejects_options():
    with pytest.raises(g.GbfftError):
        g.fft_plan_dry_run(1024, 1, radix=3)
    with pytest.raises(g.GbfftError):
        g.fft_plan_dry_run(1024, 1, schedule=0x333)     # 8*8*8 != 1024
    with pytest.raises(g.GbfftError):
        g.fft_plan_dry_run(1024, 1, precision=9)
    # tensor-core classes: 2^4 .. 2^24 on the tcgen05 kernel (six-step above
    # 2^14), 16 / 256 / 4096 on the warp-level MMA kernel (variant 1)
    for n, variant in ((2 ** 25, 0), (8, 0), (1024, 1)):
        with pytest.raises(g.GbfftError) as e:
            g.fft_plan_dry_run(n, 1, precision=g.FFT_PREC_TC_BF16, variant=variant)
        assert e.value.status == g.FFT_ERR_NOT_IMPLEMENTED
    with pytest.raises(g.GbfftError) as e:
        g.fft_plan_dry_run(1024, 1, precision=g.FFT_PREC_TC_BF16, variant=2)
    assert e.value.status == g.FFT_ERR_INVALID_ARG
    for logn in range(4, 15):
        d = g.fft_plan_dry_run(2 ** logn, 5, precision=g.FFT_PREC_TC_BF16X3)
        (p,) = d["passes"]
        assert p["tc_prec"] == 3 and 1 << sum(r.bit_length() - 1 for r in p["radices"]) == 2 ** logn
        first = [2 ** (logn % 4)] if logn % 4 else []   # FP32 first stage, then radix 16
        assert p["radices"] == first + [16] * (logn // 4) and p["smem"] <= 232448
    # complex32 storage: the tcgen05 FP16 kernel at the same lengths, nothing else
    for logn in range(4, 15):
        (p,) = g.fft_plan_dry_run(2 ** logn, 5, precision=g.FFT_PREC_TC_FP16_C32)["passes"]
        assert p["tc_prec"] == g.FFT_PREC_TC_FP16 and p["io16"] == 1
    for n, variant in ((2 ** 25, 0), (8, 0), (4096, 1)):
        with pytest.raises(g.GbfftError) as e:
            g.fft_plan_dry_run(n, 1, precision=g.FFT_PREC_TC_FP16_C32, variant=variant)
        assert e.value.status == g.FFT_ERR_NOT_IMPLEMENTED
    with pytest.raises(g.GbfftError) as e:
        g.fft_plan_dry_run(1024, 1, precision=g.FFT_PREC_TC_FP16_C32 + 1)
    assert e.value.status == g.FFT_ERR_INVALID_ARG


@pytest.mark.parametrize("logn", range(15, 25))
@pytest.mark.parametrize("precision", [1, 3, 4])
def test_tc_six_step_plans(logn, precision):
    """Tensor-core plans above 2^14: transpose, tensor-core rows of N1, transpose
    with the twiddle, rows of N2, transpose (N = N1 N2, N1 <= N2), through two
    workspace buffers, in sub-batches of at most 2^28 elements."""
    N, batch = 2 ** logn, 3
    d = g.fft_plan_dry_run(N, batch, precision=precision)
    kinds = [p["kind"] for p in d["passes"]]
    assert kinds == ["transpose", "fft", "transpose", "fft", "transpose"]
    t1, f1, t2, f2, t3 = d["passes"]
    n1, n2 = 2 ** (logn // 2), 2 ** (logn - logn // 2)
    assert (t1["rows"], t1["cols"], t1["twiddle_logN"]) == (n1, n2, 0)
    assert (t2["rows"], t2["cols"], t2["twiddle_logN"]) == (n2, n1, logn)
    assert (t3["rows"], t3["cols"], t3["twiddle_logN"]) == (n1, n2, 0)
    assert f1["L"] == n1 and f1["count_inner"] == batch * n2
    assert f2["L"] == n2 and f2["count_inner"] == batch * n1
    io16 = 1 if precision == 4 else 0
    assert all(p["io16"] == io16 for p in d["passes"])
    # in -> work -> work -> work2 -> work2 -> out
    assert [(p["src"], p["dst"]) for p in d["passes"]] == [(0, 2), (2, 2), (2, 3), (3, 3), (3, 1)]
    assert d["workspace_bytes"] == 2 * batch * N * 8
    big = g.fft_plan_dry_run(N, (2 ** 28 // N) * 2 + 1, precision=precision)
    assert big["chunk_batch"] == 2 ** 28 // N
    assert big["workspace_bytes"] == 2 * 2 ** 28 * 8


@pytest.mark.parametrize("logn", range(0, 25))
@pytest.mark.parametrize("batch", [1, 3, 64])
def test_planner_limits(logn, batch):
    """Every planned pass respects the device limits and covers its transforms."""
    smem = 232448
    d = g.fft_plan_dry_run(2 ** logn, batch, smem_optin_bytes=smem)
    assert d["max_block_log2"] == 14
    passes = d["passes"]
    assert len(passes) == (1 if logn <= 14 else 2)
    for p in passes:
        if p["kind"] != "fft":
            continue
        assert p["block"] <= 1024 and p["smem"] <= smem
        assert 1 << sum(r.bit_length() - 1 for r in p["radices"]) == p["L"]
        assert max(p["radices"]) <= p["R"]
        assert p["tiles_inner"] * p["G"] >= p["count_inner"]
    if logn > 14:
        chunk = max(1, 2 ** 28 // 2 ** logn)
        assert d["workspace_bytes"] == 8 * min(batch, chunk) * 2 ** logn
        assert d["chunk_batch"] == (chunk if batch > chunk else 0)
        p1, p2 = passes
        assert p1["L"] * p2["L"] == 2 ** logn and p1["epi"] == 4 and p2["smap"] == "cols"


def test_sar_frame_plan():
    d = g.fft_plan_dry_run((4096, 8192), 1)
    rows, cols = d["passes"]
    assert rows["L"] == 8192 and rows["count_inner"] == 4096
    assert cols["L"] == 4096 and cols["lmap"] == "cols" and cols["src"] == cols["dst"] == 1
    assert d["workspace_bytes"] == 0


def test_smaller_device_forces_more_passes():
    d = g.fft_plan_dry_run(2 ** 14, 1, smem_optin_bytes=48 * 1024)
    assert d["max_block_log2"] == 12 and len(d["passes"]) == 2


def test_conv_plan_shapes():
    """SAR compression: range pass over contiguous rows, azimuth pass over
    strided columns in place, both fused forward/filter/inverse passes."""
    d = g.fft_conv_plan_dry_run((4096, 8192), 2, [(8192, 1.0 / 4096), (1, 1.0 / 8192)])
    assert d["conv"] == 1 and d["workspace_bytes"] == 0
    rg, az = d["passes"]
    assert rg["L"] == 8192 and rg["lmap"] == rg["smap"] == "rows" and rg["h_dim"] == 1
    assert rg["h_lines"] == 1 and rg["conj_in"] == 0 and rg["conj_out"] == 1
    assert az["L"] == 4096 and az["lmap"] == az["smap"] == "cols" and az["h_dim"] == 0
    assert az["h_lines"] == 8192 and az["src"] == az["dst"] == 1
    for logn in range(1, 15):
        p = g.fft_conv_plan_dry_run(2 ** logn, 3, [(3, 1.0)])["passes"][0]
        assert p["conv"] == 1 and p["smem"] > 0 and p["block"] <= 1024
        assert len(p["radices"]) >= min(2, logn)


@pytest.mark.parametrize("n,batch,filters,status", [
    ((2 ** 15,), 1, [(1, 1.0)], g.FFT_ERR_NOT_IMPLEMENTED),
    ((1,), 1, [(1, 1.0)], g.FFT_ERR_UNSUPPORTED_SIZE),
    ((12,), 1, [(1, 1.0)], g.FFT_ERR_UNSUPPORTED_SIZE),
    ((64,), 4, [(2, 1.0)], g.FFT_ERR_INVALID_ARG),
    ((64,), 4, [(0, 1.0)], g.FFT_ERR_INVALID_ARG),
    ((16, 32), 1, [(16, 1.0), (1, 1.0)], g.FFT_ERR_INVALID_ARG),   # columns filter: 1 or 32
    ((16, 32), 1, [(32, 1.0), (32, 1.0)], g.FFT_ERR_INVALID_ARG),  # rows filter: 1 or 16
    ((16, 32), 1, [(1, float("nan")), (1, 1.0)], g.FFT_ERR_INVALID_ARG)])
def test_conv_dry_run_rejects(n, batch, filters, status):
    with pytest.raises(g.GbfftError) as e:
        g.fft_conv_plan_dry_run(n, batch, filters)
    assert e.value.status == status


@pytest.mark.parametrize("logn,split,g1,g2", [(20, 10, 8, 8), (21, 10, 8, 4), (22, 11, 4, 4),
                                              (24, 12, 4, 4), (16, 8, 16, 16)])
def test_four_step_tile_widths(logn, split, g1, g2):
    """Transforms per tile of the four-step passes: 8 at 1024 points and 4 at
    2048 and 4096 (256-thread blocks, two per SM, for 1024 and 2048), 16 for
    shorter passes; the tile option narrows them."""
    d = g.fft_plan_dry_run(2 ** logn, 4)
    p1, p2 = d["passes"]
    assert p1["L"] == 2 ** split and (p1["G"], p2["G"]) == (g1, g2)
    d = g.fft_plan_dry_run(2 ** logn, 4, tile=2)
    assert [p["G"] for p in d["passes"]] == [min(2, g1), min(2, g2)]


@pytest.mark.parametrize("logn,batch", [(22, 64), (22, 65), (22, 256), (20, 1024), (24, 17), (15, 9000)])
def test_two_pass_sub_batches(logn, batch):
    """Two-pass plans run batches above 2^28 elements in sub-batches of
    max(1, 2^28 / N) transforms and hold one sub-batch of workspace."""
    d = g.fft_plan_dry_run(2 ** logn, batch)
    chunk = max(1, 2 ** 28 // 2 ** logn)
    assert d["chunk_batch"] == (chunk if batch > chunk else 0)
    assert d["workspace_bytes"] == 8 * min(batch, chunk) * 2 ** logn
