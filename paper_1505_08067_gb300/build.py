"""Build ``libgbfft.so`` in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into one shared
library beside this file (``paper_1505_08067_gb300/lib/libgbfft.so``).  The
library's exported symbols are exactly the C ABI of ``include/gbfft.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(OUT_DIR, "libgbfft.so")
MEASURE = os.path.join(HERE, "measure")
CALL_LATENCY = os.path.join(OUT_DIR, "call_latency")  # C-side per-call timing of the ABI
SOURCES = ["kernels.cu", "generic_rows.cu", "generic_cols.cu", "generic_transposing.cu",
           "shapes_contig.cu", "shapes_fourstep.cu", "kernels_tc.cu", "kernels_umma.cu", "kernels_umma_c32.cu", "fill.cu", "conv.cu", "noalloc.cu", "queue.cu", "transpose.cu", "selftest.cu", "api.cpp",
           "exec.cpp", "server.cpp",
           "planner.cpp", "autotune.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbfft.so")


def build_id() -> str:
    """Hash of the library's sources and header: the autotune results kept in
    a GBFFT_WISDOM file are keyed by it, so a changed library tunes again."""
    import hashlib
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    with open(os.path.join(ROOT, "include", "gbfft.h"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:12]


def _flags(src: str) -> list[str]:
    f = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    if src == "autotune.cpp":
        f.append(f'-DGBFFT_BUILD_ID="{build_id()}"')
    if src.endswith(".cu"):
        f += ["-Xptxas", "-warn-spills"]
    else:
        f += ["-x", "cu"]  # host-only files still include CUDA runtime headers
    return f


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths += [os.path.join(MEASURE, f) for f in os.listdir(MEASURE)]
    paths.append(os.path.join(ROOT, "include", "gbfft.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    newest = _newest_input()
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest
            and os.path.exists(CALL_LATENCY) and os.path.getmtime(CALL_LATENCY) >= newest):
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    objdir = os.path.join(OUT_DIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    exe = nvcc()

    def compile_one(src: str) -> str:
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [exe] + _flags(src) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    # the C timing program of the small-call path links the library just built
    tmp = CALL_LATENCY + f".tmp{os.getpid()}"
    cmd = [exe] + ARCH + ["-O2", "-std=c++17", "-I" + os.path.join(ROOT, "include"),
                          os.path.join(MEASURE, "call_latency.cu"), "-o", tmp, "-L" + OUT_DIR,
                          "-lgbfft", "-Xlinker", "-rpath,$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"call_latency build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CALL_LATENCY)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
