"""Loader for the scheduler harness (test infrastructure, see sched_harness.cpp)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(os.path.dirname(HERE)), "paper_1505_08067_gb300", "csrc")
LIB = os.path.join(HERE, "_sched.so")
SRC = os.path.join(HERE, "sched_harness.cpp")
_lib = None


def load():
    global _lib
    if _lib is None:
        deps = [SRC, os.path.join(CSRC, "scheduler.h")]
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(p) for p in deps):
            tmp = LIB + f".tmp{os.getpid()}"
            subprocess.run(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-I" + CSRC, "-o", tmp,
                            SRC], check=True)
            os.replace(tmp, LIB)
        _lib = ctypes.CDLL(LIB)
        _lib.sched_simulate.restype = ctypes.c_int
    return _lib


def simulate(key, nbytes, arrive, dur, groupable, budget, max_group=256, backfill=False):
    n = len(key)
    a = lambda v, t: np.ascontiguousarray(np.asarray(v), dtype=t)
    key, arrive, dur, grp = a(key, np.int32), a(arrive, np.int32), a(dur, np.int32), a(groupable, np.int32)
    nbytes = a(nbytes, np.uint64)
    launch, gid, done, rej = (np.zeros(n, np.int32) for _ in range(4))
    peak = ctypes.c_uint64()
    p = lambda x: x.ctypes.data_as(ctypes.c_void_p)
    steps = load().sched_simulate(n, p(key), p(nbytes), p(arrive), p(dur), p(grp),
                                  ctypes.c_uint64(budget), max_group, int(backfill), p(launch),
                                  p(gid), p(done),
                                  ctypes.byref(peak), p(rej))
    return dict(steps=steps, launch=launch, group=gid, done=done, rejected=rej.astype(bool),
                peak=peak.value)
