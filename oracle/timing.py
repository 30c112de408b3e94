"""Times the FP64 CPU oracle on the rising-bubble workload (Sec. 4.4 set-up,
1024 x 4096) on the host cores, for the CPU baseline of the benchmark.

TEST INFRASTRUCTURE: run only by ``bench.py``'s CPU legs, as a child process, so
that the thread count (OMP_NUM_THREADS) and the build (LBM_ORACLE_BUILD) are
fixed before the oracle library loads. Prints one JSON line:

    python -m oracle.timing [--seconds S]

The sample is whole-grid steps of the full workload for about S seconds (one
untimed step first), or, where one full step takes longer than S / 2, steps of a
full-width horizontal slab of it (walls in y) sized to about S / 4 a step.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def omp_threads() -> int:
    """Threads the OpenMP runtime of the loaded oracle will use."""
    try:
        return int(ctypes.CDLL("libgomp.so.1").omp_get_max_threads())
    except OSError:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def measure(seconds: float) -> dict:
    from oracle import oracle as orc
    from paper_1902_08933_gb300 import workloads as wl
    orc.build()
    full = wl.rising_bubble()
    cfg = full
    P = orc.params(cfg)
    st = orc.init(P, wl.initial_phi(cfg))
    t0 = time.perf_counter()
    orc.step(P, st, 1)
    t_step = time.perf_counter() - t0
    if t_step > seconds / 2:
        rows = max(16, min(full["ny"], int(full["ny"] * (seconds / 4) / t_step)))
        cfg = dict(full, ny=rows, init=dict(full["init"], cy=rows / 2.0))
        P = orc.params(cfg)
        st = orc.init(P, wl.initial_phi(cfg))
        t0 = time.perf_counter()
        orc.step(P, st, 1)
        t_step = time.perf_counter() - t0
    n = max(1, int(seconds / max(t_step, 1e-9)))
    t0 = time.perf_counter()
    orc.step(P, st, n)
    dt = time.perf_counter() - t0
    cells = cfg["nx"] * cfg["ny"]
    what = "full 1024 x 4096 steps" if cfg is full else "steps of a 1024 x %d slab" % cfg["ny"]
    return {"mlups": cells * n / dt / 1e6, "threads": omp_threads(), "steps": n, "seconds": dt,
            "cells": cells, "build": "gcc -O3" if orc.TIMED else "gcc -O2 -ffp-contract=off",
            "sample": "%d %s (%.1f s), FP64" % (n, what, dt)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=12.0)
    args = ap.parse_args()
    print(json.dumps(measure(args.seconds)))


if __name__ == "__main__":
    main()
