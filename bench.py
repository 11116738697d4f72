#!/usr/bin/env python
"""Benchmark of the batched complex FFT on GB300.

Workload: batched 1D complex64 FFTs, N = 2^8 .. 2^14 with N * batch = 2^27
(1 GiB in, 1 GiB out per launch), forward and inverse, out-of-place, FP32.
One step = the whole sweep: 7 sizes x 2 directions = 14 transforms of 2^27
elements.  Metric: FFT GFLOP/s with the 5 N log2 N convention (Bergach et al.
Eq. 1 convention), whole job; beside it the achieved HBM bandwidth of the
Stockham pass kernel against the measured copy bandwidth (16 bytes per element
per pass: one read and one write).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): independent replicas, no collective on
the data path; value = all ranks' work / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FFT GFLOP/s (5NlogN) + % HBM roofline, FP32 vs TC mixed; served p99 latency"
LOGS = list(range(8, 15))
TOTAL_LOG = 27
DIRS = (-1, +1)
WORKLOAD = ("batched 1D complex64 FFT sweep N=2^8..2^14, N*batch=2^27 (1 GiB in) per launch, "
            "forward and inverse, out-of-place, FP32")
KERNEL_SOURCES = ["paper_1505_08067_gb300/csrc/" + f for f in (
    "fft_core.h", "fft_stage.h", "fft_split.h", "kernels_impl.cuh", "kernel_shapes.h", "kernels.cu",
    "shapes_contig.cu", "shapes_fourstep.cu", "generic_rows.cu", "generic_cols.cu",
    "generic_transposing.cu")]


def flops_of(logn: int, elements: int) -> float:
    return 5.0 * elements * logn


def step_flops(elements: int) -> float:
    return sum(flops_of(l, elements) for l in LOGS) * len(DIRS)


def kernel_source_sha() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def load_traffic(sha: str):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_sha") != sha:
        return None
    return d.get("bytes_per_launch_full_size")


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[2], parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def gpu_id_of(dev) -> str:
    """nvidia-smi id (UUID) of a torch device, "0" if unknown."""
    import torch
    try:
        props = torch.cuda.get_device_properties(dev)
        if getattr(props, "uuid", None) is not None:
            u = str(props.uuid)
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    return "0"


# ------------------------------------------------------------- replicas ----

def replica_throughput(local_ms: float, units_per_rank: float, world: int, device=None) -> tuple:
    """Whole-job throughput of independent replicas: every rank did
    `units_per_rank` units in `local_ms`; the job takes as long as the slowest
    rank.  Returns (max_ms over ranks, all ranks' units / that time per second).
    With world > 1 this is the only collective (one max all-reduce of a scalar,
    outside the timed region)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


# --------------------------------------------------------------- oracle ----

def oracle_gflops(seconds: float, steps: int = 1):
    """Times the FP64 oracle (as it stands) on a bounded sample of the workload
    sized for about `seconds` of CPU work in total over `steps` steps.
    Returns (GFLOP/s, threads, sample description, per-step sample elems)."""
    import numpy as np

    from oracle import oracle
    from paper_1505_08067_gb300 import synth
    threads = oracle.num_threads(0)
    probe = synth.uniform(2, 1, 2 ** 20).reshape(-1, 1024)
    t0 = time.perf_counter()
    oracle.fft(probe, -1)
    rate = flops_of(10, 2 ** 20) / max(time.perf_counter() - t0, 1e-6)
    per_step = seconds * rate / max(steps, 1)
    elems = 2 ** int(max(14, min(TOTAL_LOG, math.floor(math.log2(per_step / step_flops(1))))))
    x = synth.uniform(2, 1, elems)[0]
    return rate, threads, elems, x


def run_oracle_steps(x, elems, steps, warmup):
    from oracle import oracle
    for it in range(warmup + steps):
        if it == warmup:
            t0 = time.perf_counter()
        for lg in LOGS:
            for d in DIRS:
                oracle.fft(x.reshape(-1, 2 ** lg), d)
    return time.perf_counter() - t0


def reference_arm(args, rank: int, world: int = 1) -> None:
    if rank != 0:
        return
    _, threads, elems, x = oracle_gflops(60.0, args.steps + args.warmup)
    secs = run_oracle_steps(x, elems, args.steps, args.warmup)
    value = step_flops(elems) * args.steps / secs / 1e9
    sample = (f"{elems} elements (of 2^27) per size and direction per step, iid U[-1,1] "
              f"complex64 widened to FP64")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(args, world),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ ours ----

def _tuned(plan):
    t = plan.describe().get("tuning")
    if not t:
        return None
    return t.get("chosen") or t.get("cached")


def _model_record(plan, n: int, batch: int):
    """The autotuner's model step for a single-pass plan (Sec. 3.2): the
    shortest path over the measured per-(radix, start stage) costs, its
    predicted cost per element, and the whole-pass times the runtime
    validation measured on the trial batch: the default schedule's (the
    first candidate) and the model's (a candidate of its own only where it
    differs from the default; otherwise the two are the same plan)."""
    from paper_1505_08067_gb300 import gbfft
    t = plan.describe().get("tuning") or {}
    m = t.get("model")
    if not m:
        return None
    cands = t.get("candidates") or []
    default_ms = cands[0]["ms"] if cands else None
    model_ms = None
    for c in cands[1:]:
        if c["opts"].get("schedule"):
            model_ms = c["ms"]
    default = gbfft.fft_plan_dry_run(n, batch)["passes"][0]["radices"]
    return {"model_schedule": m["schedule"], "predicted_ns_per_element": m["cost_ns_per_element"],
            "default_schedule": default, "model_equals_default": model_ms is None,
            "timed_ms_default": default_ms,
            "timed_ms_model": default_ms if model_ms is None else model_ms,
            "trial_batch": t.get("trial_batch"),
            "chosen_radices": plan.describe()["passes"][0]["radices"],
            "chosen": t.get("chosen")}


def _free_device_memory():
    import gc

    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


SECTION_DESC = {
    "tc6": ("tensor-core classes above 2^14 (six-step plans: transposes and tcgen05 row "
            "passes) beside the FP32 four-step path: N=2^20 batch 64, N=2^22 batch 16, "
            "N=2^24 batch 4 (2^26 elements each), forward and inverse; FP16, BF16, split "
            "BF16x3 and FP16 with complex32 storage"),
    "multipass": ("large multi-pass 1D complex64 FFTs: N=2^20 batch 64, N=2^22 batch 16, "
                  "N=2^24 batch 4 (2^26 elements each), forward and inverse, FP32"),
    "sar": ("2D SAR frame 4096 azimuth x 8192 range complex64 (LFM chirp echoes BT=500, "
            "50 scatterers, SNR 10 dB), row then column FFTs, forward and inverse, FP32"),
    "tc": ("batched 1D complex64 FFT N=4096 batch=32768 (2^27 elements, uniform plus a "
           "1e-3 tone), and N=8192 / 16384 on the same 2^27 elements: FP32 path and the "
           "tensor-core classes FP16, BF16, split BF16x3 (tcgen05 kernel; at N=4096 also the "
           "warp-level MMA kernel) and FP16 with complex32 storage (the same input rounded to "
           "FP16 pairs, 4 B per element), forward and inverse"),
}
TC_BOUNDS = {"tc_fp16": 2e-3, "tc_bf16": 2e-3, "tc_bf16x3": 5e-6 * 12, "tc_fp16_c32": 2e-3}
PREC_C32 = 4  # FFT_PREC_TC_FP16_C32: complex32 input and output


def _to_c32(x):
    """complex64 device tensor -> complex32 (FP16 pairs, round to nearest even)."""
    import torch
    return torch.view_as_real(x).to(torch.float16).contiguous().view(torch.complex32).reshape(x.shape)


def _c32_to_numpy(y):
    """complex32 device tensor -> complex128 NumPy array of the same shape."""
    import numpy as np
    import torch
    f = y.reshape(-1).view(torch.float16).float().cpu().numpy().astype(np.float64)
    return (f[0::2] + 1j * f[1::2]).reshape(tuple(y.shape))


def section_items(kind: str, args, x_reuse=None) -> dict:
    """Multi-pass 1D (cfg3), the 2D SAR frame (cfg3) or the tensor-core class
    (cfg4): every item forward and inverse per step; per item the median
    CUDA-event time of its launch sequence and its fraction of the HBM
    roofline at 16 B per element per pass.  Clocks are sampled during the
    timed steps."""
    import numpy as np
    import torch

    from paper_1505_08067_gb300 import gbfft, synth

    if kind == "tc":
        items = [((4096,), 2 ** (TOTAL_LOG - 12)), ((8192,), 2 ** (TOTAL_LOG - 13)),
                 ((16384,), 2 ** (TOTAL_LOG - 14))]
    elif kind in ("multipass", "tc6"):
        items = [((2 ** 20,), 64), ((2 ** 22,), 16), ((2 ** 24,), 4)]
    else:
        items = [((4096, 8192), 1)]
    if args.only:
        items = [it for it in items if int(np.log2(np.prod(it[0]))) == args.only] or items
    dev = torch.device("cuda", torch.cuda.current_device())
    E = max(int(np.prod(s)) * b for s, b in items)
    tone_bins = None
    if kind == "sar":
        x = torch.from_numpy(synth.sar_frame(31).reshape(-1)).to(dev)
        data = "synth.sar_frame seed 31"
    elif kind == "tc":
        xt, tone_bins = synth.buried_tone(4, E // 4096, 4096)
        x = torch.from_numpy(xt.reshape(-1)).to(dev)
        del xt
        data = "synth.buried_tone seed 4 (iid U[-1,1] plus a 1e-3 tone at a seeded bin)"
    elif x_reuse is not None and x_reuse.numel() >= E:
        x = x_reuse[:E]
        data = "iid U[-1,1) from the device generator (the headline's seed-2 input, first 2^26 elements)"
    else:
        x = torch.empty(E, dtype=torch.complex64, device=dev)
        gbfft.fft_fill_uniform(x.data_ptr(), E, 3, 0, torch.cuda.current_stream().cuda_stream)
        data = "iid U[-1,1) from the device generator, seed 3"
    y = torch.empty_like(x)
    # complex32 copies of the input and an output for the FP16 class with
    # complex32 storage (made before the timed region)
    tc_kinds = ("tc", "tc6")
    x16 = _to_c32(x) if kind in tc_kinds else None
    y16 = torch.empty_like(x16) if kind in tc_kinds else None
    plans, order = {}, []
    # (precision, variant): FP32, the tcgen05 classes, and at N = 4096 the
    # warp-level MMA classes beside them
    precs = [(0, 0), (1, 0), (2, 0), (3, 0), (PREC_C32, 0)] if kind in tc_kinds else [(0, 0)]
    t_plan = time.perf_counter()
    for shape, batch in items:
        extra = [(1, 1), (2, 1), (3, 1)] if kind == "tc" and shape == (4096,) else []
        for prec, var in precs + extra:
            for d in DIRS:
                opts = {"epilogue": args.epilogue} if args.epilogue else {}
                if args.variant and prec == 0:
                    opts["variant"] = args.variant
                if prec:
                    opts["variant"] = var
                if args.tile and prec == 0:
                    opts["tile"] = args.tile
                opts["autotune"] = args.autotune if prec == 0 else 0
                key = (shape, d, prec, var)
                plans[key] = gbfft.Plan(shape if len(shape) > 1 else shape[0], batch, d, prec,
                                        **opts)
                order.append((key, int(np.prod(shape)) * batch, int(np.log2(np.prod(shape)))))
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()

    def io(key):  # the buffers of an item: complex32 for that class
        return (x16, y16) if key[2] == PREC_C32 else (x, y)

    def esz(key):  # bytes per stored element
        return 4 if key[2] == PREC_C32 else 8

    for _ in range(args.warmup):
        for key, e, _lg in order:
            xi, yi = io(key)
            plans[key].execute(xi[:e], yi[:e], stream)
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in order] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_id_of(dev))
    sampler.start()
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    bnd = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")
    a.record(stream)
    for s in range(args.steps):
        for i, (key, e, _lg) in enumerate(order):
            xi, yi = io(key)
            ev[s][i][0].record(stream)
            plans[key].execute(xi[:e], yi[:e], stream)
            ev[s][i][1].record(stream)
    bnd.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = sampler.stop()
    ms = a.elapsed_time(bnd)
    flops = sum(5.0 * e * lg for _k, e, lg in order)
    peaks = load_peaks()
    per = {}
    for i, (key, e, lg) in enumerate(order):
        t = statistics.median(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
        passes = len(plans[key].describe()["passes"])
        pname = PREC_NAMES[key[2]] + ("_warp_mma" if key[3] == 1 else "")
        # bytes of the algorithm (one read and one write per pass of an FP32
        # two-pass plan: 2 passes above 2^14), not of the six-step transposes
        alg_passes = min(passes, 2)
        gbs = 2.0 * esz(key) * alg_passes * e / (t * 1e-3) / 1e9
        per[f"{'x'.join(map(str, key[0]))} {'fwd' if key[1] < 0 else 'inv'} {pname}"] = {
            "ms": round(t, 4), "gflops": round(5.0 * e * lg / (t * 1e-3) / 1e9, 1),
            "passes": passes, "gbs": round(gbs, 1), "frac": round(gbs / peaks["hbm_gbs"], 4),
            "tuned": _tuned(plans[key])}
    tot_bytes = sum(2.0 * esz(k) * min(len(plans[k].describe()["passes"]), 2) * e
                    for k, e, _ in order)
    launches = sum(plans[k].launch_count for k, _e, _l in order) * args.steps
    out = {
        "workload": SECTION_DESC[kind], "data": data, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "gflops": flops * args.steps / (ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                     "achieved": round(tot_bytes * args.steps / (ms * 1e-3) / 1e9, 1),
                     "frac": round(tot_bytes * args.steps / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                     "alg_bytes": "16 B per element per pass (8 B for complex32 storage)"},
        "per_item": per, "clocks": clocks, "gpu_launches": launches,
        "plan_create_s": round(t_plan, 2),
        "l2": "inputs of 256 MiB to 1 GiB per launch, larger than L2; no flush"}
    if kind == "tc6":
        out["roofline"]["alg_bytes"] = ("16 B per element per pass of the two-pass algorithm (8 B "
                                        "for complex32), the six-step plans' five passes counted "
                                        "as two")
        out["accuracy_vs_fp32"] = _six_step_accuracy(gbfft, x)
        out["vs_fp32"] = {
            "x".join(map(str, shape)): {
                p: {d: round(per[f"{shape[0]} {d} fp32"]["ms"] / per[f"{shape[0]} {d} {p}"]["ms"], 3)
                    for d in ("fwd", "inv")}
                for p in ("tc_fp16", "tc_bf16", "tc_bf16x3", "tc_fp16_c32")}
            for shape, _b in items}
    if kind == "tc":
        acc = _tc_accuracy(gbfft, x, tone_bins)
        for name, rec in acc.items():
            rec["bound"] = TC_BOUNDS[name.replace("_warp_mma", "")]
            rec["within_bound"] = rec["rel_l2_max"] <= rec["bound"]
        out["accuracy_vs_fp32"] = acc
        # time ratio FP32 / class per length and direction (> 1: the class is faster)
        vs = {}
        for shape, _b in items:
            nm = "x".join(map(str, shape))
            fp32 = {d: per[f"{nm} {d} fp32"]["ms"] for d in ("fwd", "inv")}
            names = ["tc_fp16", "tc_bf16", "tc_bf16x3", "tc_fp16_c32"]
            if shape == (4096,):
                names += ["tc_fp16_warp_mma", "tc_bf16_warp_mma", "tc_bf16x3_warp_mma"]
            vs[nm] = {p: {d: round(fp32[d] / per[f"{nm} {d} {p}"]["ms"], 3) for d in ("fwd", "inv")}
                      for p in names}
        out["vs_fp32"] = vs
    for p in plans.values():
        p.close()
    del x, y, x16, y16
    return out


PREC_NAMES = ["fp32", "tc_fp16", "tc_bf16", "tc_bf16x3", "tc_fp16_c32"]


SIX_STEP_BOUNDS = {"tc_fp16": lambda n: 2e-3, "tc_bf16": lambda n: 7e-3,
                   "tc_bf16x3": lambda n: 5e-6 * math.log2(n), "tc_fp16_c32": lambda n: 2e-3}


def _six_step_accuracy(gbfft, x) -> dict:
    """Relative L2 error of each tensor-core class's six-step plan against this
    library's FP32 four-step path (1e-7 level against the FP64 oracle in the
    parity tests) on the first transform of the input, at 2^20 and 2^24.  The
    complex32 form reads the input rounded to FP16 pairs, so its error includes
    that rounding."""
    import numpy as np
    import torch

    acc = {}
    for logn in (20, 24):
        n = 2 ** logn
        xs = x[:n]
        with gbfft.Plan(n, 1, -1) as p:
            ref = p.execute(xs).cpu().numpy().astype(np.complex128)
        for prec, name in ((1, "tc_fp16"), (2, "tc_bf16"), (3, "tc_bf16x3"), (PREC_C32, "tc_fp16_c32")):
            with gbfft.Plan(n, 1, -1, prec) as p:
                if prec == PREC_C32:
                    y = _c32_to_numpy(p.execute(_to_c32(xs)))
                else:
                    y = p.execute(xs).cpu().numpy().astype(np.complex128)
                torch.cuda.synchronize()
            e = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
            bound = SIX_STEP_BOUNDS[name](n)
            acc[f"{n} {name}"] = {"rel_l2": e, "bound": bound, "within_bound": e <= bound}
    return acc


def _tc_accuracy(gbfft, x, bins, count: int = 64, n: int = 4096, amplitude: float = 1e-3):
    """Error of each tensor-core class on the first `count` transforms of the
    tone-bearing input, against this library's FP32 path (itself 2-5e-7 from the
    FP64 oracle in the parity tests): max and mean relative L2 per transform, and
    the error at each transform's tone bin relative to the tone's exact
    contribution n * amplitude.  The complex32 class reads the input rounded to
    FP16 pairs, so its error includes that rounding."""
    import numpy as np
    import torch

    xs = x[:count * n]
    outs = {}
    for prec, var in ((0, 0), (1, 0), (2, 0), (3, 0), (PREC_C32, 0), (1, 1), (2, 1), (3, 1)):
        name = PREC_NAMES[prec] + ("_warp_mma" if var == 1 else "")
        with gbfft.Plan(n, count, -1, prec, **({"variant": var} if prec else {})) as p:
            if prec == PREC_C32:
                outs[name] = _c32_to_numpy(p.execute(_to_c32(xs))).reshape(count, n)
            else:
                outs[name] = p.execute(xs).cpu().numpy().reshape(count, n).astype(np.complex128)
            torch.cuda.synchronize()
    ref = outs.pop("fp32")
    k0 = np.asarray(bins[:count])
    acc = {}
    for name, y in outs.items():
        rel = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
        tone = np.abs(y[np.arange(count), k0] - ref[np.arange(count), k0]) / (n * amplitude)
        acc[name] = {"rel_l2_max": float(rel.max()), "rel_l2_mean": float(rel.mean()),
                     "tone_err_max": float(tone.max()), "transforms": count}
    return acc


def section_serve(args, jobs: int, load: float) -> dict:
    """Serving (cfg5): a Poisson stream of FFT jobs, sizes log-uniform over
    N = 2^8..2^22, batch 1..256, forward / inverse 50/50, 80% FP32 and 20%
    tensor-core class (log-uniform over 2^8 .. 2^serve_tc_max_log: single-pass
    up to 2^14, six-step above), admitted under a 64 GB budget.  Offered load: algorithmic bytes
    per second = `load` x measured HBM bandwidth.  Inputs are slices of one
    seeded device buffer; outputs rotate through a ring that is reused only
    after the job holding it completes.  Reports p50/p99 latency and aggregate
    GFLOP/s (5 N log2 N of completed jobs over the wall time of the stream)."""
    import threading
    from collections import deque

    import numpy as np
    import torch

    from paper_1505_08067_gb300 import gbfft, synth

    rng = np.random.default_rng(5)
    njobs = jobs
    logn = rng.integers(8, 23, njobs)
    batch = rng.integers(1, 257, njobs)
    dirs = np.where(rng.random(njobs) < 0.5, -1, 1)
    prec = np.where(rng.random(njobs) < 0.2, rng.integers(1, 4, njobs), 0)
    # tensor-core jobs: log-uniform over 2^8 .. 2^serve_tc_max_log
    logn = np.where(prec > 0, rng.integers(8, args.serve_tc_max_log + 1, njobs), logn)
    elems = (2 ** logn) * batch
    passes = np.where(logn > 14, 2, 1)
    alg_bytes = 16.0 * passes * elems
    peaks = load_peaks()
    rate = load * peaks["hbm_gbs"] * 1e9 / alg_bytes.mean()            # jobs per second
    gaps = rng.exponential(1.0 / rate, njobs)
    dev = torch.device("cuda", torch.cuda.current_device())
    in_elems = 1 << 30                                                 # 8 GiB of inputs
    xin = torch.empty(in_elems, dtype=torch.complex64, device=dev)
    gbfft.fft_fill_uniform(xin.data_ptr(), in_elems, 5, 0, torch.cuda.current_stream().cuda_stream)
    ring_elems = 6 << 30                                               # 48 GiB of outputs
    yout = torch.empty(ring_elems, dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    srv = gbfft.fft_server_create(memory_budget_bytes=64 * 10 ** 9, streams=args.streams,
                                  strict_order=int(args.strict_order),
                                  large_group_log2=args.large_group_log2)
    # warm the plans of every key outside the measured stream
    keys = sorted(set(zip(logn.tolist(), dirs.tolist(), prec.tolist())))
    for lg, d, p in keys:
        t = gbfft.fft_server_submit(srv, 2 ** lg, 1, d, p, xin.data_ptr(), yout.data_ptr())
        gbfft.fft_server_wait(srv, t)
    outstanding = deque()          # (ticket, ring start, ring end)
    lock = threading.Lock()
    results = []
    done_flag = threading.Event()
    errors = []

    def waiter():
        try:
            while True:
                with lock:
                    item = outstanding[0] if outstanding else None
                if item is None:
                    if done_flag.is_set():
                        return
                    time.sleep(0.0002)
                    continue
                r = gbfft.fft_server_wait(srv, item[0])
                results.append(r)
                with lock:
                    outstanding.popleft()
        except BaseException as exc:  # surfaced by the main thread
            errors.append(repr(exc))
            done_flag.set()

    base_stats = gbfft.fft_server_stats(srv)
    sampler = ClockSampler(gpu_id_of(dev))
    sampler.start()
    th = threading.Thread(target=waiter)
    th.start()
    ring = 0
    ring_waits = 0
    t0 = time.perf_counter()
    t_next = t0
    for j in range(njobs):
        need = int(elems[j])
        if ring + need > ring_elems:
            ring = 0
        waited = False
        while True:                 # the ring slice must be free
            with lock:
                busy = any(not (ring + need <= s or ring >= e) for _, s, e in outstanding)
            if not busy or errors:
                break
            waited = True
            time.sleep(0.0002)
        ring_waits += waited
        t_next += gaps[j]
        while time.perf_counter() < t_next:
            pass
        src = int(rng.integers(0, in_elems - need + 1)) & ~1
        t = gbfft.fft_server_submit(srv, 2 ** int(logn[j]), int(batch[j]), int(dirs[j]),
                                    int(prec[j]), xin.data_ptr() + 8 * src,
                                    yout.data_ptr() + 8 * ring)
        with lock:
            outstanding.append((t, ring, ring + need))
        ring += need
    t_sub = time.perf_counter() - t0
    done_flag.set()
    th.join()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    if errors:
        raise RuntimeError("serving waiter failed: " + errors[0])
    stats = gbfft.fft_server_stats(srv)
    gbfft.fft_server_destroy(srv)
    lat = np.array([r["latency_ms"] for r in results if r["status"] == 0])
    queue = np.array([r["queue_ms"] for r in results if r["status"] == 0])
    ok = sum(r["status"] == 0 for r in results)
    status_counts = {}
    for r in results:
        status_counts[str(r["status"])] = status_counts.get(str(r["status"]), 0) + 1
    flops = float(np.sum(5.0 * elems * logn))
    offered_s = float(np.sum(gaps))
    del xin, yout
    return {
        "workload": "serving: Poisson stream of FFT jobs, N = 2^8..2^22 (tensor-core jobs "
                    f"N = 2^8..2^{args.serve_tc_max_log}), batch 1..256, 50/50 forward/inverse, "
                    "80% FP32 / 20% tensor-core class, 64 GB budget",
        "alg_bytes": "16 B per element per pass, two passes above 2^14 (the six-step "
                     "tensor-core plans move more: five passes)",
        "jobs": njobs, "offered_load_frac_of_hbm": load, "offered_jobs_per_s": rate,
        "streams": args.streams, "large_group_log2": args.large_group_log2,
        "admission": "strict arrival order" if args.strict_order else "backfilling",
        "tc_share": float((prec > 0).mean()), "mean_job_elements": float(elems.mean()),
        "gflops": flops / wall / 1e9,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()), "max": float(lat.max())},
        "queue_ms": {"p50": float(np.percentile(queue, 50)), "p99": float(np.percentile(queue, 99))},
        "completed": int(ok), "waited": len(results), "status_counts": status_counts,
        "submit_s": t_sub, "offered_s": offered_s, "wall_s": wall,
        "submitter_ring_waits": int(ring_waits),
        "offered_alg_gbs": float(alg_bytes.sum() / offered_s / 1e9),
        "achieved_alg_gbs": float(alg_bytes.sum() / wall / 1e9),
        "achieved_frac_of_hbm": float(alg_bytes.sum() / wall / 1e9 / peaks["hbm_gbs"]),
        "all_offered_served": bool(wall <= offered_s * 1.05 and ok == njobs),
        "clocks": clocks,
        "server": {k: stats[k] - base_stats.get(k, 0) if k in ("launches", "groups",
                   "coalesced_jobs", "completed", "backfilled_jobs", "host_launch_s",
                   "group_stream_s") else stats[k]
                   for k in ("launches", "groups", "coalesced_jobs", "completed",
                             "backfilled_jobs", "peak_bytes_in_flight",
                             "workspace_allocations", "host_launch_s", "group_stream_s")}}


def section_compress(args) -> dict:
    """SAR range + azimuth compression of one 4096 (azimuth) x 8192 (range)
    raw frame: two fused convolution passes (forward FFT, matched filter,
    inverse FFT per line), the azimuth pass with one filter per range bin.
    Flops: forward and inverse 2D FFT, 2 x 5 N log2 N with N = 2^25 (the
    filter products are not counted).  Algorithmic bytes: 16 B per element
    for the range pass (its one filter stays in L2), 24 B for the azimuth pass
    (per-line filters are a frame-sized array).  The range pass alone is timed
    too (a 1D convolution plan over the same rows runs the same kernel)."""
    import numpy as np
    import torch

    from paper_1505_08067_gb300 import gbfft, synth

    rows, cols = 4096, 8192
    E = rows * cols
    dev = torch.device("cuda", torch.cuda.current_device())
    frame, rr, az, _pos = synth.sar_raw(31, rows, cols)
    x = torch.from_numpy(frame.reshape(-1)).to(dev)
    y = torch.empty_like(x)
    # matched-filter spectra conj(DFT(replica)) with the library's own FFTs
    with gbfft.Plan(cols, 1, -1) as p:
        hr = p.execute(torch.from_numpy(rr).to(dev)).conj().resolve_conj().contiguous()
    az_t = torch.from_numpy(np.ascontiguousarray(az.T)).to(dev)          # (cols, rows)
    with gbfft.Plan(rows, cols, -1) as p:
        ha = p.execute(az_t.reshape(-1)).reshape(cols, rows).t().conj().resolve_conj().contiguous()
    del az_t
    vopt = {"variant": args.variant} if args.variant else {}
    full = gbfft.ConvPlan((rows, cols), 1, [(ha.reshape(-1), cols, 1.0 / rows),
                                            (hr, 1, 1.0 / cols)], **vopt)
    rng_only = gbfft.ConvPlan(cols, rows, [(hr, 1, 1.0 / cols)], **vopt)
    stream = torch.cuda.current_stream()

    def timed(plan, steps):
        for _ in range(args.warmup):
            plan.execute(x, y, stream)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            plan.execute(x, y, stream)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / steps

    sampler = ClockSampler(gpu_id_of(dev))
    sampler.start()
    ms_full = timed(full, args.steps)
    ms_rng = timed(rng_only, args.steps)
    clocks = sampler.stop()
    ms_az = max(ms_full - ms_rng, 1e-6)
    # end to end: pinned host frame in, compressed frame out
    h_in = torch.from_numpy(frame.reshape(-1)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    full.execute_host(h_in, h_out, x, y, stream)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    k2 = max(1, min(args.steps, args.e2e_steps))
    a.record(stream)
    for _ in range(k2):
        full.execute_host(h_in, h_out, x, y, stream)
    b.record(stream)
    torch.cuda.synchronize()
    ms_e2e = a.elapsed_time(b) / k2
    flops = 2 * 5.0 * E * math.log2(E)
    peaks = load_peaks()
    g_rng = 16.0 * E / (ms_rng * 1e-3) / 1e9
    g_az = 24.0 * E / (ms_az * 1e-3) / 1e9
    full.close()
    rng_only.close()
    del x, y, hr, ha
    return {
        "workload": "SAR range + azimuth compression, 4096 x 8192 complex64 frame, "
                    "per-range-bin azimuth filters",
        "data": "synthetic: 50 point scatterers, LFM range chirp BT=500, range-dependent "
                "azimuth chirps of 512 samples, SNR 10 dB (seed 31)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_frame": ms_full,
        "frames_per_s": 1e3 / ms_full, "gflops": flops / (ms_full * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                     "kernel": "stockham_staged, convolution form (azimuth pass)", "achieved": round(g_az, 1),
                     "frac": round(g_az / peaks["hbm_gbs"], 4), "alg_bytes_per_launch": 24.0 * E},
        "passes": {"range": {"ms": round(ms_rng, 4), "gbs": round(g_rng, 1),
                             "frac": round(g_rng / peaks["hbm_gbs"], 4), "alg_bytes": 16.0 * E},
                   "azimuth": {"ms": round(ms_az, 4), "gbs": round(g_az, 1),
                               "frac": round(g_az / peaks["hbm_gbs"], 4), "alg_bytes": 24.0 * E}},
        "e2e": {"value": flops / (ms_e2e * 1e-3) / 1e9, "unit": "GFLOP/s",
                "h2d_bytes_per_step": 8 * E, "d2h_bytes_per_step": 8 * E,
                "api": "fft_execute_host"},
        "clocks": clocks, "gpu_launches": 2 * args.steps,
        "l2": "frame and azimuth filters 256 MiB each, larger than L2; no flush"}


def section_cufft(args) -> dict:
    """Context only (not the product path): the same transforms through
    torch.fft, i.e. cuFFT on this GPU, beside this library, on the same
    device-resident inputs with the same timing (CUDA events on the launching
    stream, median of the timed repetitions after warm-up): the sweep sizes
    2^8..2^14 on 2^27 elements, the two-pass sizes 2^20 / 2^22 / 2^24 on 2^26
    elements, the 4096 x 8192 frame (2D) and N = 1024 x 64, forward.  Inputs of
    256 MiB and up exceed L2 (no flush); the small case is L2-resident for
    both."""
    import numpy as np
    import torch

    from paper_1505_08067_gb300 import gbfft
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    items = ([((2 ** e,), 2 ** (TOTAL_LOG - e)) for e in range(8, 15)] +
             [((2 ** e,), 2 ** (26 - e)) for e in (20, 22, 24)] + [((4096, 8192), 1), ((1024,), 64)])
    E = max(int(np.prod(sh)) * b for sh, b in items)
    x = torch.empty(E, dtype=torch.complex64, device=dev)
    gbfft.fft_fill_uniform(x.data_ptr(), E, 5, 0, stream.cuda_stream)
    y = torch.empty_like(x)
    reps, warm = max(args.steps // 2, 10), 3

    def timed(fn):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for a, b in ev:
            a.record(stream)
            fn()
            b.record(stream)
        torch.cuda.synchronize()
        return statistics.median(a.elapsed_time(b) for a, b in ev)

    peaks = load_peaks()
    per = {}
    sampler = ClockSampler(gpu_id_of(dev))
    sampler.start()
    for shape, batch in items:
        e = int(np.prod(shape)) * batch
        xi, yi = x[:e], y[:e]
        if len(shape) == 1:
            xv = xi.view(batch, shape[0])
            ref = lambda: torch.fft.fft(xv, dim=-1)  # noqa: E731
        else:
            xv = xi.view(batch, *shape)
            ref = lambda: torch.fft.fft2(xv)  # noqa: E731
        with gbfft.Plan(shape if len(shape) > 1 else shape[0], batch, -1) as p:
            ours = timed(lambda: p.execute(xi, yi, stream))
            passes = len(p.describe()["passes"])
        cu = timed(ref)
        lg = int(np.log2(np.prod(shape)))
        key = f"{'x'.join(map(str, shape))} x {batch}"
        byts = 16.0 * passes * e
        per[key] = {"ours_ms": round(ours, 4), "cufft_ms": round(cu, 4),
                    "speedup_vs_cufft": round(cu / ours, 3),
                    "ours_gflops": round(5.0 * e * lg / (ours * 1e-3) / 1e9, 1),
                    "cufft_gflops": round(5.0 * e * lg / (cu * 1e-3) / 1e9, 1),
                    "ours_frac": round(byts / (ours * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    clocks = sampler.stop()
    torch.cuda.empty_cache()  # cuFFT plans and torch.fft outputs
    return {"workload": "context: torch.fft (cuFFT, torch " + torch.__version__ + ") beside "
                        "fft_execute on the same inputs, forward, complex64",
            "data": "iid U[-1,1) from the device generator, seed 5", "reps": reps,
            "warmup": warm, "per_item": per, "clocks": clocks,
            "note": "cuFFT is a comparator for context; no part of this library calls it"}


def section_small(args) -> dict:
    """Small batch (cfg1): N = 1024, batch 64 (512 KiB), launch-latency bound.
    Per call of fft_execute (one kernel launch), fft_execute_graph (the same
    launch replayed from a CUDA graph) and fft_execute_noalloc: measured from
    C by the library's call_latency program (host enqueue time, device time
    back to back, and the median round trip of single synchronised calls,
    beside an empty kernel's; and the persistent work queue's round trip of a
    submit and a wait, and its time per job back to back), and through this
    Python binding."""
    import torch

    from paper_1505_08067_gb300 import build as gbuild
    from paper_1505_08067_gb300 import gbfft, synth
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(synth.uniform(1, 64, 1024)).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    py = {}
    with gbfft.Plan(1024, 64, -1) as p:
        for name, fn in (("fft_execute", p.execute), ("fft_execute_graph", p.execute_graph)):
            for _ in range(20):
                fn(x, y, stream)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            reps = 2000
            t0 = time.perf_counter()
            a.record(stream)
            for _ in range(reps):
                fn(x, y, stream)
            b_.record(stream)
            torch.cuda.synchronize()
            host = (time.perf_counter() - t0) / reps * 1e6
            dev_us = a.elapsed_time(b_) / reps * 1e3
            py[name] = {"device_us": round(dev_us, 3), "host_us": round(host, 3),
                        "gflops": round(5.0 * 1024 * 10 * 64 / (dev_us * 1e-6) / 1e9, 1)}
    del x, y
    c = None
    if not os.path.exists(gbuild.CALL_LATENCY):
        raise RuntimeError(f"{gbuild.CALL_LATENCY} is missing: build the package first")
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = env.get("CUDA_VISIBLE_DEVICES", str(torch.cuda.current_device()))
    r = subprocess.run([gbuild.CALL_LATENCY, "1024", "64", "2000"], capture_output=True,
                       text=True, timeout=300)
    if r.returncode != 0:
        raise RuntimeError(f"call_latency failed ({r.returncode}): {r.stderr.strip()[-400:]}")
    c = json.loads(r.stdout.strip().splitlines()[-1])
    return {"workload": "N=1024 batch 64 complex64 forward (512 KiB), calls back to back on "
                        "one stream", "from_c": c, "through_python_ctypes": py}


def headline_config(args, world: int) -> dict:
    return {"workload": WORKLOAD, "sizes": [2 ** l for l in LOGS],
            "elements_per_launch": 2 ** TOTAL_LOG, "precision": "FP32",
            "l2": "inputs larger than L2 (1 GiB per launch), no flush",
            "autotune": bool(args.autotune), "variant": args.variant,
            "parallelism": "replicas" if world > 1 else "single GPU"}


def ours(args, rank: int, world: int) -> None:
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1505_08067_gb300 import gbfft, synth

    dev = torch.device("cuda", torch.cuda.current_device())
    E = 2 ** TOTAL_LOG
    # seeded uniform noise generated on the device (counter-based hash; the
    # same values as synth.uniform_hash(2, E))
    x = torch.empty(E, dtype=torch.complex64, device=dev)
    gbfft.fft_fill_uniform(x.data_ptr(), E, 2, 0, torch.cuda.current_stream().cuda_stream)
    y = torch.empty_like(x)
    plans = {}
    for lg in LOGS:
        for d in DIRS:
            opts = {"autotune": args.autotune}
            if args.variant:
                opts["variant"] = args.variant
            plans[(lg, d)] = gbfft.Plan(2 ** lg, E >> lg, d, **opts)
    launches_per_step = sum(p.launch_count for p in plans.values())
    stream = torch.cuda.current_stream()
    order = [(lg, d) for lg in LOGS for d in DIRS]

    def one_step(evs=None):
        for i, key in enumerate(order):
            if evs is not None:
                evs[i][0].record(stream)
            plans[key].execute(x, y, stream)
            if evs is not None:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    sampler = ClockSampler(gpu_id_of(dev))
    sampler.start()
    ev = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in order]
          for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed_steps")  # lets ncu select the timed launches only
    start.record(stream)
    for s in range(args.steps):
        one_step(ev[s])
    end.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = start.elapsed_time(end)
    per_launch = {key: [] for key in order}
    for s in range(args.steps):
        for i, key in enumerate(order):
            per_launch[key].append(ev[s][i][0].elapsed_time(ev[s][i][1]))
    ms_max, flops_per_s = replica_throughput(ms, step_flops(E) * args.steps, world, dev)
    ms_per_step = ms_max / args.steps
    value = flops_per_s / 1e9

    # roofline of the Stockham pass kernel (every launch here is one pass)
    peaks = load_peaks()
    alg_bytes = 16.0 * E
    all_ms = [v for vs in per_launch.values() for v in vs]
    avg_ms = sum(all_ms) / len(all_ms)
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    sha = kernel_source_sha()
    traffic = load_traffic(sha)
    per_size = {}
    model = {}
    for lg in LOGS:
        tms = statistics.median(per_launch[(lg, -1)] + per_launch[(lg, +1)])
        per_size[f"2^{lg}"] = {"ms": round(tms, 4),
                               "gflops": round(flops_of(lg, E) / (tms * 1e-3) / 1e9, 1),
                               "gbs": round(alg_bytes / (tms * 1e-3) / 1e9, 1),
                               "frac": round(alg_bytes / (tms * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                               "radices": plans[(lg, -1)].describe()["passes"][0]["radices"],
                               "tuned": _tuned(plans[(lg, -1)])}
        rec = _model_record(plans[(lg, -1)], 2 ** lg, E >> lg)
        if rec:
            model[f"2^{lg}"] = rec

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        h_in = torch.empty(x.shape, dtype=x.dtype, pin_memory=True)
        h_in.copy_(x)
        h_out = torch.empty_like(h_in).pin_memory()

        def e2e_step():
            for key in order:
                plans[key].execute_host(h_in, h_out, x, y, stream)
        e2e_step()
        torch.cuda.synchronize()
        k2 = max(1, min(args.steps, args.e2e_steps))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        a.record(stream)
        for _ in range(k2):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        t2 = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        e2e = {"value": world * step_flops(E) * k2 / (float(t2.item()) * 1e-3) / 1e9,
               "unit": "GFLOP/s", "h2d_bytes_per_step": 8 * E * len(order),
               "d2h_bytes_per_step": 8 * E * len(order), "steps": k2,
               "api": "fft_execute_host (pinned host buffers, chunked H2D/kernel/D2H overlap)",
               "host_numa": host_numa_record(dev)}
        del h_in, h_out
    for p in plans.values():
        p.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        _, threads, elems, xs = oracle_gflops(15.0, 1)
        secs = run_oracle_steps(xs, elems, 1, 0)
        cpu = {"value": step_flops(elems) / secs / 1e9, "unit": "GFLOP/s", "cores": threads,
               "kind": "oracle",
               "sample": f"one sweep step on {elems} of the 2^27 elements per size and direction"}

    configs = None
    if args.sections and world == 1:
        configs = {}
        x_keep = x
        del y
        _free_device_memory()
        for name in args.sections:
            t0 = time.perf_counter()
            try:
                if name == "small":
                    rec = section_small(args)
                elif name == "multipass":
                    rec = section_items("multipass", args, x_keep)
                elif name == "sar":
                    rec = section_items("sar", args)
                elif name == "tc":
                    rec = section_items("tc", args)
                elif name == "tc6":
                    rec = section_items("tc6", args)
                elif name == "serve":
                    rec = section_serve(args, args.serve_jobs, args.load)
                elif name == "serve_tc14":
                    # the same stream with tensor-core jobs up to 2^14 only (single-pass)
                    a14 = argparse.Namespace(**vars(args))
                    a14.serve_tc_max_log = 14
                    rec = section_serve(a14, args.serve_jobs, args.load)
                elif name == "sar_compress":
                    rec = section_compress(args)
                elif name == "cufft":
                    rec = section_cufft(args)
                else:
                    rec = {"error": f"unknown section {name}"}
            except Exception as exc:  # recorded in the line, not hidden
                rec = {"error": f"{type(exc).__name__}: {exc}"}
            rec["section_s"] = round(time.perf_counter() - t0, 1)
            configs[SECTION_KEYS.get(name, name)] = rec
            if name == "multipass":
                x_keep = None
            _free_device_memory()
    elif args.sections:
        configs = {"skipped": "the per-configuration sections run at n_gpus = 1 only"}

    if rank == 0:
        frac = achieved / peaks["hbm_gbs"]
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: iid U[-1,1) complex64 from a counter-based hash (SplitMix64, "
                    "seed 2), generated on the device (fft_fill_uniform)",
            "config": headline_config(args, world),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(frac, 4),
                         "traffic": traffic, "kernel": "stockham_pass",
                         "alg_bytes_per_launch": alg_bytes,
                         "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)"},
            "pct_hbm_roofline": round(100 * frac, 2),
            "per_size": per_size,
            "autotune_model": model,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
        }
        if configs is not None:
            line["configs"] = configs
        print(json.dumps(line))


SECTION_KEYS = {"small": "cfg1_small_call", "multipass": "cfg3_multipass", "sar": "cfg3_sar_frame",
                "tc": "cfg4_tensor_core", "tc6": "cfg4_tensor_core_six_step", "serve": "cfg5_serving",
                "serve_tc14": "cfg5_serving_tc_single_pass", "sar_compress": "sar_compression",
                "cufft": "context_cufft"}
DEFAULT_SECTIONS = "small,multipass,sar,tc,tc6,serve,serve_tc14,sar_compress,cufft"


def host_numa_record(dev) -> dict:
    """Where the pinned host buffers of the e2e leg live relative to the GPU:
    the NUMA node the GPU's PCI/C2C device reports, the nodes this process may
    allocate on, and the CPUs it runs on (read from sysfs and procfs; nothing is
    changed)."""
    rec = {}
    try:
        import torch
        props = torch.cuda.get_device_properties(dev)
        bus = getattr(props, "pci_bus_id", None)
        dom = getattr(props, "pci_domain_id", None)
        devid = getattr(props, "pci_device_id", None)
        if bus is not None:
            addr = f"{dom or 0:04x}:{bus:02x}:{devid or 0:02x}.0"
            p = f"/sys/bus/pci/devices/{addr}/numa_node"
            rec["gpu_pci"] = addr
            if os.path.exists(p):
                rec["gpu_numa_node"] = int(open(p).read().strip())
    except Exception as exc:
        rec["gpu_error"] = str(exc)
    try:
        for line in open("/proc/self/status"):
            if line.startswith(("Mems_allowed_list", "Cpus_allowed_list")):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
    except Exception:
        pass
    try:
        nodes = sorted(d for d in os.listdir("/sys/devices/system/node") if d.startswith("node"))
        rec["host_numa_nodes"] = nodes
    except Exception:
        pass
    return rec


def main() -> None:
    global LOGS, TOTAL_LOG
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--jobs", type=int, default=20000, help="serve workload: number of jobs")
    ap.add_argument("--load", type=float, default=0.5,
                    help="serve workload: offered algorithmic bytes/s as a fraction of HBM")
    ap.add_argument("--streams", type=int, default=4, help="serve workload: server streams")
    ap.add_argument("--large-group-log2", type=int, default=0,
                    help="serve workload: groups of at least 2^k elements run in order on the "
                         "first stream (0: library default, -1: any stream)")
    ap.add_argument("--strict-order", action="store_true",
                    help="serve workload: admit strictly in arrival order (no backfilling)")
    ap.add_argument("--workload", choices=["sweep", "multipass", "sar", "tc", "tc6", "serve", "small", "cufft",
                                           "sar_compress"],
                    default="sweep",
                    help="sweep: the headline batched N=2^8..2^14 line with every other "
                         "configuration as a section; the others: one configuration alone")
    ap.add_argument("--autotune", type=int, default=1)
    ap.add_argument("--only", type=int, default=0, help="run only N = 2^ONLY (profiling)")
    ap.add_argument("--tile", type=int, default=0,
                    help="multipass / sar workloads: transforms per tile (0: library choice)")
    ap.add_argument("--variant", type=int, default=0,
                    help="contiguous-pass kernel variant (0 library choice, 1 register, "
                         "2 TMA-staged, 3 L2 prefetch)")
    ap.add_argument("--epilogue", type=int, default=0,
                    help="four-step twiddle source for two-pass plans (0 library choice)")
    ap.add_argument("--total-log", type=int, default=TOTAL_LOG,
                    help="log2 of elements per launch (profiling of smaller cases)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sections", default=DEFAULT_SECTIONS,
                    help="sweep workload: comma-separated per-configuration sections timed after "
                         "the headline and reported under 'configs' (small, multipass, sar, tc, "
                         "serve, sar_compress), or 'none'")
    ap.add_argument("--serve-tc-max-log", type=int, default=22,
                    help="serving: largest log2 N of the tensor-core jobs (14: single-pass only)")
    ap.add_argument("--serve-jobs", type=int, default=4000,
                    help="jobs of the serving section of the sweep workload")
    args = ap.parse_args()
    args.sections = [] if args.sections in ("", "none") else args.sections.split(",")
    if args.warmup < 3:
        args.warmup = 3
    if args.only:
        LOGS = [args.only]
    TOTAL_LOG = args.total_log
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload == "sweep":
        ours(args, rank, world)
    else:
        # one configuration alone, printed as its own line (not the headline)
        if args.workload == "serve":
            rec = section_serve(args, args.jobs, args.load)
        elif args.workload == "small":
            rec = section_small(args)
        elif args.workload == "sar_compress":
            rec = section_compress(args)
        elif args.workload == "cufft":
            rec = section_cufft(args)
        else:
            rec = section_items(args.workload, args)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "n_gpus": world, "section": args.workload,
                              **rec}))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
