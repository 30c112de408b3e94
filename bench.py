#!/usr/bin/env python
"""Benchmark: MLUPS and fraction of the HBM roofline of the fused phase-field
lattice Boltzmann step (arXiv:1902.08933, Sec. 3) on one GB300, with FP64, FP32,
FP16-storage and batched forms side by side, their error against FP64, the
end-to-end rate through the C ABI with host buffers, and the FP64 CPU oracle
timed on the host cores.

Workload (headline): rising bubble, 1024 x 4096, bounce-back walls in y,
periodic x, R = 128 at y = 512, density ratio 10, Eo = 10, Re = 35, W = 5,
quasi-incompressible model, pressure of Eq. 28; FP32 storage and arithmetic with
h_0 kept as a two-float pair (form LBM_F32_C: the fastest FP32 form, and the one
that conserves sum(phi) to round-off). One step = one lattice time step of the
whole grid (both population sets). The state (2 x 369 MB ping-pong) is larger
than the 129 MB L2, so no L2 flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own independent replica of the
workload (weak scaling, no data-path collective) for the headline value; the
line also carries the 512 mixed instances split by instance across the ranks
and the 1024 x 4096 bubble split into slabs with a ghost-row exchange over NCCL
(both strong scaling). Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# bytes each storage form moves a lattice update (state read once and written once)
BYTES_PER_LUP = {"f64": 336, "f32": 168, "f32_g16": 140, "f32_h16": 108, "f32_c": 176, "f32_cc": 176}
# the method's algorithmic bytes: 9 + 9 populations, phi u (2) and p read and
# written once in the form's word size; the two-float h_0 of f32_c (8 bytes, not
# 4) is the form's own addition and not counted
ALGO_BYTES_PER_LUP = {"f64": 336, "f32": 168, "f32_c": 168, "f32_cc": 168, "f32_g16": 132, "f32_h16": 100}
# D3Q15: 15 + 15 populations, phi u (3), p, each read and written once
BYTES_PER_LUP_D3 = {"f64": 544, "f32": 272, "f32_c": 280}
METRIC = "MLUPS and % of HBM peak, FP64 vs FP32/FP16-storage vs batched, at stated error"
L2_BYTES = 129e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="f32_c", choices=list(BYTES_PER_LUP))
    ap.add_argument("--pipeline", default="auto",
                    choices=["auto", "plain", "async", "tma", "pairs", "batched", "persistent"],
                    help="load path / kernel of the step (lbm_set_pipeline); also for --kernel-run on "
                         "the D3Q15 bubble (async: the fused march, plain: the three-kernel step) and "
                         "the batched instances")
    ap.add_argument("--kernel-run", default=None,
                    choices=["bubble3d", "source_flow", "source_flow_remark1", "source_flow_remark2",
                             "source_flow_remark4", "batched"],
                    help="only time one step loop of another workload (for profiling): the "
                         "128 x 256 x 128 D3Q15 bubble, the 4096 x 4096 single-phase source "
                         "flow of Remark 3, Remark 1 or the Remark 4 scheme with drag, or the "
                         "512 mixed instances of the batched configuration")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the side-by-side forms, e2e and CPU legs")
    ap.add_argument("--no-tune", action="store_true",
                    help="time the built-in launch plan instead of the autotuner's choice "
                         "(profiling runs: no trial launches before the timed ones)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.1)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------- helpers
def traffic_record(kernel_key):
    """DRAM bytes per step from the committed ncu summary (key: the storage form,
    plus "/persistent" for the several-steps-a-launch kernel, whose launch is
    divided by the steps it ran), if the kernel source has not changed since it
    was captured (else None)."""
    h = hashlib.sha256()
    for name in ("lbm_device.cuh", "lbm_step_x2.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1902_08933_gb300", "csrc", name), "rb").read())
    sha = h.hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", "step_kernel_bubble_1024x4096.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    t = re.search(r"traffic_bytes_per_step\[%s\]:\s*([0-9.eE+]+)" % re.escape(kernel_key), text)
    if not m or not t or m.group(1) != sha:
        return None
    return float(t.group(1))


# FP64 pipe of GB300: 2 FP64 FMA a clock per SM (the nominal 1.25 TFLOP/s at
# 152 SMs and 2.07 GHz).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PIPE_OPS_PER_S = 152 * 2 * 2.07e9


def fp64_roofline(mlups, measured_tflops=None):
    """ALU roofline of the FP64 form from the FP64 operation counts per lattice
    update in the committed ncu summary (None if absent), against the FP64 FMA
    throughput measured on this GPU (lbm_measure_fp64_fma), else the nominal."""
    path = os.path.join(ROOT, "profiles", "step_kernel_f64_bubble_1024x4096.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    flop = re.search(r"fp64_flop_per_lup:\s*([0-9.]+)", text)
    inst = re.search(r"fp64_inst_per_lup:\s*([0-9.]+)", text)
    if not flop or not inst:
        return None
    achieved = float(flop.group(1)) * mlups * 1e6 / 1e12
    peak = measured_tflops if measured_tflops else FP64_PEAK_TFLOPS
    kind = ("measured: independent FP64 FMA chains on every SM (lbm_measure_fp64_fma)" if measured_tflops
            else "nominal: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_kind": kind, "nominal_peak": FP64_PEAK_TFLOPS,
            "fp64_pipe_frac": float(inst.group(1)) * mlups * 1e6 / (peak * 1e12 / 2)}


def rel_err(a, b):
    import numpy as np
    den = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def warm(sim, n):
    """n warm-up steps in one call: a call of two or more steps also captures the
    step graph, so no capture falls inside a timed region."""
    if n > 0:
        sim.step(n)
    sim.sync()


def time_steps(lbm, sim, stream, steps, warmup):
    import torch
    warm(sim, warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


# ------------------------------------------------------------------------- CPU oracle
def oracle_rate(threads, seconds):
    """FP64 oracle (its -O3 timed build) on the host cores, in a child process
    with OMP_NUM_THREADS = threads: whole 1024 x 4096 steps for about `seconds`
    (a full-width slab where one step is too long). Returns oracle.timing's record."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), LBM_ORACLE_BUILD="timed")
    r = subprocess.run([sys.executable, "-m", "oracle.timing", "--seconds", str(seconds)],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: %s" % r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands (its -O3 timed build) on the
    host cores, each step one whole time step of the 1024 x 4096 bubble, or of a
    full-width horizontal slab of it where the whole run would not end within
    about two minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    os.environ["LBM_ORACLE_BUILD"] = "timed"
    from oracle import oracle as orc
    from oracle import timing
    from paper_1902_08933_gb300 import workloads as wl
    orc.build()
    full = wl.rising_bubble()
    P = orc.params(full)
    st = orc.init(P, wl.initial_phi(full))
    t0 = time.perf_counter()
    orc.step(P, st, 1)
    t_step = time.perf_counter() - t0
    budget_s = 120.0
    cfg = full
    if (args.steps + args.warmup) * t_step > budget_s:
        rows = int(max(16, min(full["ny"], full["ny"] * budget_s /
                               ((args.steps + args.warmup) * t_step))))
        cfg = dict(full, ny=rows, init=dict(full["init"], cy=rows / 2.0))
        P = orc.params(cfg)
        st = orc.init(P, wl.initial_phi(cfg))
    orc.step(P, st, args.warmup)
    t0 = time.perf_counter()
    orc.step(P, st, args.steps)
    dt = time.perf_counter() - t0
    cells = cfg["nx"] * cfg["ny"]
    mlups = cells * args.steps / dt / 1e6
    threads = timing.omp_threads()
    same = cfg is full
    sample = ("%d whole 1024 x 4096 steps" % args.steps if same else
              "%d steps of a %d x %d slab of the 1024 x 4096 bubble (walls in y)" % (
                  args.steps, cfg["nx"], cfg["ny"])) + ", gcc -O3 build"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "rising_bubble_1024x4096_rho10_qim" + ("" if same else " (CPU slab sample)"),
                   "rows": cfg["ny"], "same_config": same},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ------------------------------------------------------------------------- GPU arm
def kernel_run(args):
    """Times args.steps steps of one secondary workload after args.warmup
    warm-up steps and prints one line (used to profile those kernels)."""
    import numpy as np
    import torch
    from paper_1902_08933_gb300 import build, lbm
    from paper_1902_08933_gb300 import workloads as wl
    build.build()
    stream = torch.cuda.Stream()
    if args.kernel_run == "batched":
        cfgs = wl.batched_mixed(512)
        cells = int(wl.lups(cfgs, 1))
        form = args.form
        sim = lbm.Simulation(cfgs, form, stream=stream.cuda_stream,
                             phi0=[wl.initial_phi(c) for c in cfgs])
        bpl = BYTES_PER_LUP[form]
    elif args.kernel_run == "bubble3d":
        cfg = wl.rising_bubble3()
        cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
        form = args.form if args.form in BYTES_PER_LUP_D3 else "f32_c"
        sim = lbm.Simulation(cfg, form, stream=stream.cuda_stream, phi0=[wl.initial_phi(cfg)])
        bpl = BYTES_PER_LUP_D3[form]
    else:
        n = 4096
        cells = n * n
        src = np.ascontiguousarray(1e-4 * np.sin(2 * np.pi * np.arange(n) / n)[None, :] * np.ones((n, 1)))
        form = "f64" if args.form == "f64" else "f32"
        model = {"source_flow": 0, "source_flow_remark1": 1, "source_flow_remark2": 2,
                 "source_flow_remark4": 4}[args.kernel_run]
        spcfg = dict(nx=n, ny=n, nu=0.1, model=model if model in (1, 2) else 0)
        if model == 4:
            spcfg.update(scheme=1, force_x=1e-6, drag_lin=1e-3, drag_quad=0.1)
        sim = lbm.SourceFlow(spcfg, form, stream=stream.cuda_stream, source=src)
        bpl = {0: 76, 1: 132, 2: 132, 4: 160}[model] * (2 if form == "f64" else 1)
    if args.pipeline != "auto" and args.kernel_run in ("batched", "bubble3d"):
        lbm.lbm_set_pipeline(sim.ctx, getattr(lbm, "LBM_PIPELINE_" + args.pipeline.upper()))
    shape = None
    if args.kernel_run == "batched" and not args.no_tune and args.pipeline == "auto":
        sim.step(2)
        shape = lbm.lbm_autotune_shape(sim.ctx)
    sim.step(max(args.warmup, 2))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"kernel_run": args.kernel_run, "form": form, "ms_per_step": ms,
                      "MLUPS": cells / ms / 1e3, "GBps_algorithmic": bpl * cells / ms / 1e6,
                      "launch_shape": shape}))
    sim.close()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.kernel_run:
        return kernel_run(args)
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1902_08933_gb300 import build, lbm
    from paper_1902_08933_gb300 import workloads as wl
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()

    def barrier():
        if world > 1:
            dist.barrier()

    cfg = wl.rising_bubble()
    cells = cfg["nx"] * cfg["ny"]
    phi0 = wl.initial_phi(cfg)
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()

    # ---- headline: K steps of the fused kernel, CUDA events on its stream
    sim = lbm.Simulation(cfg, args.form, stream=stream.cuda_stream, phi0=[phi0])
    lbm.lbm_set_pipeline(sim.ctx, {"auto": lbm.LBM_PIPELINE_AUTO, "plain": lbm.LBM_PIPELINE_PLAIN,
                                   "async": lbm.LBM_PIPELINE_ASYNC, "tma": lbm.LBM_PIPELINE_TMA,
                                   "pairs": lbm.LBM_PIPELINE_PAIRS, "batched": lbm.LBM_PIPELINE_BATCHED,
                                   "persistent": lbm.LBM_PIPELINE_PERSISTENT}[args.pipeline])
    shape = None
    if args.pipeline == "auto" and not args.no_tune:
        sim.step(2)
        shape = lbm.lbm_autotune_shape(sim.ctx)   # state and time level are left as they were
    launches = lbm.lbm_launches_per_step(sim.ctx)
    variant = lbm.lbm_launch_info(sim.ctx, 0)["variant"]
    warm(sim, args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = lbm.lbm_step_launch_count(sim.ctx)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    n_launches = lbm.lbm_step_launch_count(sim.ctx) - n0
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    d = sim.diagnostics()
    sim.close()
    value = world * cells * args.steps / (ms * 1e-3) / 1e6
    # per step: a launch of the persistent plan runs up to 64 steps, and its
    # algorithmic bytes over its duration is this same rate
    per_step_s = ms * 1e-3 / args.steps
    achieved = ALGO_BYTES_PER_LUP[args.form] * cells / per_step_s / 1e9
    achieved_form = BYTES_PER_LUP[args.form] * cells / per_step_s / 1e9
    persistent = (shape or {}).get("pipeline") == "persistent" or args.pipeline == "persistent"
    traffic = traffic_record(args.form + ("/persistent" if persistent else ""))
    result = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "f64" else "f32", "data": "synthetic",
        "config": {"workload": "rising_bubble_1024x4096_rho10_qim", "nx": cfg["nx"], "ny": cfg["ny"],
                   "form": args.form, "load_path": variant, "storage": {"f64": "f64", "f32": "f32",
                                                  "f32_g16": "h0 2xf32, h1-8 f32, g f16",
                                                  "f32_h16": "h0 2xf32, h1-8 f16, g f16",
                                                  "f32_c": "h0 2xf32, h1-8 f32, g f32",
                                                  "f32_cc": "h0 2xf32, h1-8 f32, g f32, "
                                                            "mu from the two-float phi"}[args.form],
                   "l2": "state %.0f MB > 129 MB L2, no flush" % (
                       2 * BYTES_PER_LUP[args.form] / 2 * cells / 1e6),
                   "parallelism": "replicas" if world > 1 else "single",
                   "launch_shape": shape if shape else {"pipeline": args.pipeline, "tuned": False}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_lup": ALGO_BYTES_PER_LUP[args.form],
                     "form_bytes_per_lup": BYTES_PER_LUP[args.form],
                     "frac_form_bytes": achieved_form / hbm_peak,
                     "kernel": "step_kernel_x2_multi" if persistent else "step_kernel_x2",
                     "per": "step (bytes of one step over one step's time; a launch runs %.1f steps)" % (
                         args.steps / max(1, n_launches))},
        "clocks": clk,
        "gpu_launches": n_launches,
        "mass_drift": abs(d["sum_phi"] - phi0.sum()) / phi0.sum(),
    }

    if world > 1 and not args.headline_only:
        result["multi_gpu"] = multi_gpu_legs(args, lbm, wl, cfg, phi0, stream, rank, world)

    if not args.headline_only and rank == 0:
        result.update(side_legs(args, lbm, wl, cfg, phi0, stream, hbm_peak))

    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def multi_gpu_legs(args, lbm, wl, cfg, phi0, stream, rank, world):
    """Under torchrun with N > 1 (one rank per GPU), besides the replicas of the
    headline: (1) the 512 mixed instances split by instance (sharding.py: no
    exchange while stepping), (2) the 1024 x 4096 bubble as N horizontal slabs
    with 12 ghost rows, exchanged over NCCL every 4 steps (slab.py). Both fix the
    total work (strong scaling); the job time is the slowest rank's."""
    import torch
    import torch.distributed as dist
    from paper_1902_08933_gb300 import sharding, slab
    out = {}
    K = max(50, args.steps // 4)

    def timed(fn):
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        dist.barrier()
        return sharding.max_over_ranks(secs, device=torch.device("cuda", torch.cuda.current_device()))

    cfgs = wl.batched_mixed(512)
    cells = [c["nx"] * c["ny"] for c in cfgs]
    mine = sharding.shard(cells, rank, world)
    with lbm.Simulation([cfgs[i] for i in mine], "f32", stream=stream.cuda_stream,
                        phi0=[wl.initial_phi(cfgs[i]) for i in mine]) as sim:
        sim.step(2)
        lbm.lbm_autotune_shape(sim.ctx)
        warm(sim, 6)
        secs = timed(lambda: sim.step(K))
    out["batched_sharded"] = {"MLUPS": sum(cells) * K / secs / 1e6, "steps": K, "scaling": "strong",
                              "instances_per_rank": len(mine),
                              "imbalance": sharding.imbalance(cells, world)}
    ghost = 12
    slabs = slab.plan(cfg["ny"], world, ghost, periodic=not cfg["walls_y"])
    me = slabs[rank]
    with torch.cuda.stream(stream), lbm.Simulation(
            slab.local_config(cfg, me, world), args.form, stream=stream.cuda_stream,
            phi0=[slab.local_field(phi0, me)]) as sim:
        run = slab.SlabRun(slabs, ghost, {rank: slab.GpuSlab(lbm, sim, 0)}, not cfg["walls_y"],
                           group=dist.group.WORLD)
        run.start()
        run.advance(2 * run.k)
        secs = timed(lambda: run.advance(K))
    out["slab"] = {"MLUPS": cfg["nx"] * cfg["ny"] * K / secs / 1e6, "steps": K, "scaling": "strong",
                   "ghost_rows": ghost, "steps_between_exchanges": ghost // slab.REACH,
                   "rows_per_rank": me.own, "form": args.form}
    return out


def side_legs(args, lbm, wl, cfg, phi0, stream, hbm_peak):
    """Other forms on the same workload, their error against FP64 on the GPU after
    the same steps, the batched mixed-size configuration, the end-to-end rate
    through the C ABI with host buffers, and the CPU oracle."""
    import numpy as np
    import torch
    out = {}
    cells = cfg["nx"] * cfg["ny"]
    K = max(50, args.steps // 4)
    acc_steps = 200
    ref = None
    forms = {}
    fp64_peak = lbm.lbm_measure_fp64_fma(stream.cuda_stream)
    for form in ("f64", "f32", "f32_c", "f32_cc", "f32_g16", "f32_h16"):
        with lbm.Simulation(cfg, form, stream=stream.cuda_stream, phi0=[phi0]) as sim:
            sim.step(acc_steps)
            f = sim.fields(0, ("phi", "ux", "uy", "p"))
            if form == "f64":
                ref = f
            shape = lbm.lbm_autotune_shape(sim.ctx)
            ms = time_steps(lbm, sim, stream, K, 5)
            mlups = cells * K / (ms * 1e-3) / 1e6
            gbs = BYTES_PER_LUP[form] * cells / (ms * 1e-3 / K) / 1e9
            forms[form] = {"MLUPS": mlups, "GBps": gbs, "frac_hbm": gbs / hbm_peak,
                           "frac_hbm_algorithmic": ALGO_BYTES_PER_LUP[form] * cells / (ms * 1e-3 / K) / 1e9 / hbm_peak,
                           "steps": K, "launch_shape": shape,
                           "kernel": lbm.lbm_launch_info(sim.ctx, 0)["variant"],
                           "roofline": fp64_roofline(mlups, fp64_peak) if form == "f64" else
                           {"bound": "hbm", "frac": gbs / hbm_peak},
                           "err_vs_f64_after_%d_steps" % acc_steps: (
                               None if form == "f64" else
                               {k: rel_err(f[k], ref[k]) for k in ("phi", "ux", "uy", "p")})}
    out["forms"] = forms

    # the three load paths of the FP32 step kernel on the headline workload
    pipes = {}
    for name, mode in (("plain", lbm.LBM_PIPELINE_PLAIN), ("async", lbm.LBM_PIPELINE_ASYNC),
                       ("tma", lbm.LBM_PIPELINE_TMA), ("pairs", lbm.LBM_PIPELINE_PAIRS)):
        with lbm.Simulation(cfg, "f32", stream=stream.cuda_stream, phi0=[phi0]) as sim:
            lbm.lbm_set_pipeline(sim.ctx, mode)
            ms = time_steps(lbm, sim, stream, K, 5)
            gbs = BYTES_PER_LUP["f32"] * cells / (ms * 1e-3 / K) / 1e9
            pipes[name] = {"MLUPS": cells * K / (ms * 1e-3) / 1e6, "frac_hbm": gbs / hbm_peak,
                           "blocks": lbm.lbm_launch_info(sim.ctx, 0)["blocks"]}
    out["f32_load_paths"] = pipes

    # batched: 512 independent droplets / bubbles of mixed size, at the autotuned
    # shape (which may be several launch classes run as concurrent graph
    # branches) and as the one persistent launch a step (the batched kernel's
    # built-in plan); 128 steps: whole graph replays from an even parity
    cfgs = wl.batched_mixed(512)
    lups_per_step = wl.lups(cfgs, 1)
    batched = {}
    for form in ("f32", "f32_g16", "f32_h16", "f32_c"):
        with lbm.Simulation(cfgs, form, stream=stream.cuda_stream,
                            phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
            Kb = 128
            sim.step(2)
            shape = lbm.lbm_autotune_shape(sim.ctx)
            ms = time_steps(lbm, sim, stream, Kb, 6)
            batched[form] = {"MLUPS": lups_per_step * Kb / (ms * 1e-3) / 1e6,
                             "launches_per_step": lbm.lbm_launches_per_step(sim.ctx),
                             "variant": lbm.lbm_launch_info(sim.ctx, 0)["variant"],
                             "launch_shape": shape}
            lbm.lbm_set_pipeline(sim.ctx, lbm.LBM_PIPELINE_BATCHED)
            lbm.lbm_set_launch(sim.ctx, 0, 0)
            ms1 = time_steps(lbm, sim, stream, Kb, 6)
            batched[form]["one_launch"] = {"MLUPS": lups_per_step * Kb / (ms1 * 1e-3) / 1e6,
                                           "launches_per_step": lbm.lbm_launches_per_step(sim.ctx),
                                           "variant": lbm.lbm_launch_info(sim.ctx, 0)["variant"]}
    batched["instances"] = len(cfgs)
    batched["cells"] = int(lups_per_step)
    out["batched"] = batched

    # D3Q15: the rising bubble in 3-D, 128 x 256 x 128 (4.2 M cells), three kernels a step
    cfg3 = wl.rising_bubble3()
    phi3 = wl.initial_phi(cfg3)
    cells3 = cfg3["nx"] * cfg3["ny"] * cfg3["nz"]
    d3 = {"workload": cfg3["name"], "cells": cells3}
    for form in ("f64", "f32", "f32_c"):
        with lbm.Simulation(cfg3, form, stream=stream.cuda_stream, phi0=[phi3]) as sim:
            K3 = max(20, K // (8 if form == "f64" else 2))
            ms = time_steps(lbm, sim, stream, K3, 6)
            gbs = BYTES_PER_LUP_D3[form] * cells3 / (ms * 1e-3 / K3) / 1e9
            d3[form] = {"MLUPS": cells3 * K3 / (ms * 1e-3) / 1e6, "GBps_algorithmic": gbs,
                        "frac_hbm": gbs / hbm_peak, "steps": K3}
    out["d3q15"] = d3

    # single-phase model of Remark 3 (div u = S): 4096 x 4096, sinusoidal source
    import numpy as np
    n = 4096
    src = np.ascontiguousarray(1e-4 * np.sin(2 * np.pi * np.arange(n) / n)[None, :] * np.ones((n, 1)))
    sp = {"workload": "source_flow_4096x4096", "cells": n * n}
    # Remark 1 (two kernels a step): (9 + 1) reads + 2 writes of u, then
    # 9 + 1 + 2 reads and 9 writes, so 264 / 132 bytes a cell
    sp1 = {"workload": "source_flow_remark1_4096x4096", "cells": n * n}
    sp2 = {"workload": "source_flow_remark2_4096x4096", "cells": n * n}   # Remark 2: as Remark 1
    # Remark 4 scheme with a drag force (two kernels): 9 reads and 4 writes (u, F),
    # then 9 + 1 + 4 + 4 reads (f, S, u and F at t and t - 1) and 9 writes: 320 / 160
    sp4 = {"workload": "source_flow_remark4_drag_4096x4096", "cells": n * n}
    legs = {0: sp, 1: sp1, 2: sp2, 4: sp4}
    for model, form, bpl in ((0, "f64", 152), (0, "f32", 76), (1, "f64", 264), (1, "f32", 132),
                             (2, "f64", 264), (2, "f32", 132), (4, "f64", 320), (4, "f32", 160)):
        spcfg = dict(nx=n, ny=n, nu=0.1, model=model if model in (1, 2) else 0)
        if model == 4:
            spcfg.update(scheme=1, force_x=1e-6, drag_lin=1e-3, drag_quad=0.1)
        with lbm.SourceFlow(spcfg, form, stream=stream.cuda_stream, source=src) as sim:
            sim.step(4)
            torch.cuda.synchronize()
            Ks = max(20, K // 4)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(Ks)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            gbs = bpl * n * n / (ms * 1e-3 / Ks) / 1e9
            legs[model][form] = {"MLUPS": n * n * Ks / (ms * 1e-3) / 1e6, "GBps_algorithmic": gbs,
                                 "frac_hbm": gbs / hbm_peak, "bytes_per_lup": bpl, "steps": Ks}
    out["source_flow"] = sp
    out["source_flow_remark1"] = sp1
    out["source_flow_remark2"] = sp2
    out["source_flow_remark4"] = sp4

    # end to end through the C ABI with host buffers: init from pinned host phi0,
    # every step's record of sum(phi), the kinetic energy and max |u| (the
    # per-step monitor) written to host memory from the GPU, the fields read
    # back to the host at the end. lbm_step_monitored_all runs CH steps a call
    # and writes the CH records into one of two pinned buffers; the records of
    # call c are checked on the host while call c + 1 runs. The context takes
    # its autotuned launch shape (the persistent plan on this grid, where the
    # records come from inside the launch).
    # 500 steps at least whatever --steps is, so that the one-time phi0 upload
    # and field read-back are spread as in a real run, not over a handful of steps
    CH = 25
    Ke = max(500, args.steps // 4) // CH * CH
    pinned = torch.from_numpy(phi0).pin_memory()
    host_phi0 = pinned.numpy()
    fields_out = torch.zeros((4, cfg["ny"], cfg["nx"]), dtype=torch.float64).pin_memory().numpy()
    size = ctypes.sizeof(lbm.lbm_monitor)
    bufs = [torch.zeros(CH * size, dtype=torch.uint8).pin_memory() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def check(call):
        base = bufs[call % 2].data_ptr()
        for k in range(CH):
            r = lbm.lbm_monitor.from_address(base + k * size)
            t = call * CH + k
            if r.nonfinite or r.device_status or r.time != t:
                raise RuntimeError("monitor record of step %d: %s" % (t, (r.nonfinite, r.device_status, r.time)))
        return r

    with lbm.Simulation(cfg, args.form, stream=stream.cuda_stream) as sim:
        lbm.lbm_set_monitor(sim.ctx, True)
        lbm.lbm_init(sim.ctx, 0, host_phi0)
        shape_e2e = lbm.lbm_autotune_shape(sim.ctx)
        lbm.lbm_step_monitored_all(sim.ctx, CH, bufs[0].data_ptr())   # warm-up (launch setup)
        lbm.lbm_get_fields(sim.ctx, 0, 0xF, fields_out)   # warm-up: the context's read-back scratch is allocated once
        sim.sync()
        t0 = time.perf_counter()
        lbm.lbm_init(sim.ctx, 0, host_phi0)
        calls = Ke // CH
        last = None
        for call in range(calls):
            lbm.lbm_step_monitored_all(sim.ctx, CH, bufs[call % 2].data_ptr())
            done[call % 2].record(stream)
            if call >= 1:
                done[(call - 1) % 2].synchronize()
                check(call - 1)
        done[(calls - 1) % 2].synchronize()
        last = check(calls - 1)
        mon = {"sum_phi": last.sum_phi}
        t1 = time.perf_counter()
        lbm.lbm_get_fields(sim.ctx, 0, 0xF, fields_out)
        dt = time.perf_counter() - t0
        t_read = time.perf_counter() - t1
    # the one-time copies alone (same calls, outside the timed loop)
    with lbm.Simulation(cfg, args.form, stream=stream.cuda_stream) as sim:
        lbm.lbm_init(sim.ctx, 0, host_phi0)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        lbm.lbm_init(sim.ctx, 0, host_phi0)
        t_init = time.perf_counter() - t2
    d2h = ctypes.sizeof(lbm.lbm_monitor) + 8 * 4 * cells / Ke
    out["e2e"] = {"value": cells * Ke / dt / 1e6, "unit": "MLUPS",
                  "h2d_bytes_per_step": 8 * cells / Ke, "d2h_bytes_per_step": d2h,
                  "steps": Ke, "per_step": ("every step's record (sum phi, kinetic energy, max |u|) reduced "
                                           "by the step kernels and written into pinned host memory from the "
                                           "GPU: lbm_step_monitored_all, %d steps a call into one of two "
                                           "buffers, each call's records checked on the host while the next "
                                           "call runs; launch shape %s" % (CH, shape_e2e.get("pipeline"))),
                  "once": "lbm_init from pinned host phi0 (%.1f MB, about %.2f ms) before the first step, "
                          "lbm_get_fields of phi, ux, uy, p to pinned host memory (%.1f MB, %.2f ms) after "
                          "the last, both inside the timed region and spread over its %d steps (one "
                          "read-back in the warm-up allocates the context's read-back scratch)" % (
                              8 * cells / 1e6, t_init * 1e3, 32 * cells / 1e6, t_read * 1e3, Ke),
                  "ms_per_step_loop": (dt - t_init - t_read) * 1e3 / Ke,
                  "mass_drift_monitor": abs(mon["sum_phi"] - float(phi0.sum())) / float(phi0.sum())}

    # CPU oracle on the host cores (bounded samples of the same workload: whole-grid
    # steps for about 12 s on every core, then a single-thread figure)
    allc = oracle_rate(os.cpu_count() or 1, 12.0)
    one = oracle_rate(1, 8.0)
    out["cpu_baseline"] = {"value": allc["mlups"], "unit": "MLUPS", "cores": allc["threads"],
                           "kind": "oracle", "build": allc["build"],
                           "sample": allc["sample"] + ", OpenMP over rows",
                           "single_thread": {"value": one["mlups"], "unit": "MLUPS", "cores": 1,
                                             "sample": one["sample"]}}
    return out


if __name__ == "__main__":
    main()
