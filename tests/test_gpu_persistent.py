"""The persistent plan (LBM_PIPELINE_PERSISTENT): the paired plan's work items run
for several steps in one cooperative launch, one block per item, each block
waiting before step s only for the items within one step's reach of its own to
finish step s - 1. The per-cell arithmetic is the paired kernel's on the same
work items, so the populations must equal the per-step paired plan's bit for
bit (the paired plan is held to the oracle in test_gpu_parity.py)."""
import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FORMS = ["f32", "f32_c", "f32_cc", "f32_g16", "f32_h16"]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def cases():
    # walls with a ragged last strip and runs of both directions; periodic in
    # both directions (wrap of the neighbour lists in x and y); tiny grids, where
    # a single strip's few short runs are each other's neighbours across the
    # periodic seam, or a walled strip has just two runs
    return [(wl.rising_bubble(nx=300, ny=170, R=20, cy=55, W=4.0, Re=8.0), 31),
            (wl.static_droplet(n=128, R=30), 23),
            (wl.static_droplet(n=32, R=8.0), 17),
            (wl.rising_bubble(nx=64, ny=20, R=5.0, cy=7.0, W=4.0, Re=5.0), 19)]


def run(L, cfg, form, mode, steps, graphs=True, rows=0):
    import torch
    stream = torch.cuda.Stream()
    with L.Simulation([cfg], form, stream=stream.cuda_stream, phi0=[wl.initial_phi(cfg)]) as sim:
        L.lbm_set_pipeline(sim.ctx, mode)
        L.lbm_set_launch(sim.ctx, 0, rows)
        L.lbm_set_graphs(sim.ctx, graphs)
        for n in steps:
            sim.step(n)
        return sim.populations(0), L.lbm_launches_per_step(sim.ctx), L.lbm_launch_info(sim.ctx, 0)


@pytest.mark.parametrize("form", FORMS)
def test_persistent_equals_per_step_pairs(L, form):
    for cfg, n in cases():
        steps = (3, n, 70)   # odd counts: both buffer parities start a launch
        ref, _, _ = run(L, cfg, form, L.LBM_PIPELINE_PAIRS, steps)
        for graphs in (True, False):
            got, launches, info = run(L, cfg, form, L.LBM_PIPELINE_PERSISTENT, steps, graphs)
            assert launches == 1 and info["variant"] == "pairs"
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (form, cfg["nx"], graphs)


def test_persistent_falls_back_when_items_do_not_fit(L):
    # 8-row runs on 1024 x 1024: 4 strips x 128 runs = 512 items, more than the
    # resident blocks; the context runs the per-step paired plan instead
    cfg = wl.static_droplet(n=1024, R=200)
    ref, _, _ = run(L, cfg, "f32_c", L.LBM_PIPELINE_PAIRS, (5,), rows=8)
    got, _, _ = run(L, cfg, "f32_c", L.LBM_PIPELINE_PERSISTENT, (5,), rows=8)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)


def test_persistent_wait_timeout_is_reported_and_checkpoint_recovers(L, tmp_path):
    cfg = wl.rising_bubble(nx=256, ny=120, R=16, cy=40, W=4.0, Re=8.0)
    phi0 = wl.initial_phi(cfg)
    ckpt = str(tmp_path / "persistent.bin")
    with L.Simulation([cfg], "f32_c", phi0=[phi0]) as ref, L.Simulation([cfg], "f32_c", phi0=[phi0]) as sim:
        for s in (ref, sim):
            L.lbm_set_pipeline(s.ctx, L.LBM_PIPELINE_PERSISTENT)
        ref.step(30)
        expected = ref.populations(0)
        sim.step(10)
        L.lbm_save(sim.ctx, ckpt)
        sim.step(7)
        L.lbm_inject_batched_wait_timeout(sim.ctx, 1 << 12)
        with pytest.raises(L.LbmError) as e:
            sim.sync()
        assert e.value.status == L.LBM_ETIMEOUT
        L.lbm_load(sim.ctx, ckpt)
        sim.step(20)
        for a, b in zip(sim.populations(0), expected):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode", ["PERSISTENT", "PAIRS"])
def test_every_step_record(L, mode):
    # lbm_step_monitored_all: the record of every step, [step][instance], written
    # from the GPU -- inside the persistent launch (steps overlapping) or one
    # monitored launch a step. Each record is the step's input level: it equals
    # the diagnostics of an unmonitored run stopped there (to the rounding of a
    # different summation order), and monitoring leaves the state bit for bit.
    import ctypes
    import torch
    cfg = wl.rising_bubble(nx=256, ny=144, R=18, cy=48, W=4.0, Re=8.0)
    phi0 = wl.initial_phi(cfg)
    cells = cfg["nx"] * cfg["ny"]
    size = ctypes.sizeof(L.lbm_monitor)
    nsteps = 70                                      # more than one launch of 64
    buf = torch.zeros(nsteps * size, dtype=torch.uint8).pin_memory()
    with L.Simulation([cfg], "f32_c", phi0=[phi0]) as sim, L.Simulation([cfg], "f32_c", phi0=[phi0]) as ref:
        for s in (sim, ref):
            L.lbm_set_pipeline(s.ctx, getattr(L, "LBM_PIPELINE_" + mode))
        sim.step(5)
        ref.step(5)
        L.lbm_set_monitor(sim.ctx, True)
        L.lbm_step_monitored_all(sim.ctx, nsteps, buf.data_ptr())
        sim.sync()
        for k in range(nsteps):
            r = L.lbm_monitor.from_address(buf.data_ptr() + k * size)
            d = ref.diagnostics(0)
            assert r.time == 5 + k and r.nonfinite == 0 and r.device_status == 0, (k, r.time)
            # the bars of the monitor against the diagnostics for the FP32 forms
            # (the diagnostics recompute u in FP64 from the stored state)
            assert abs(r.sum_phi - d["sum_phi"]) <= cells * 2.0 ** -24, k
            assert abs(r.kinetic_energy - d["kinetic_energy"]) <= 1e-4 * d["kinetic_energy"], k
            assert abs(r.max_u - d["max_u"]) <= 1e-4 * d["max_u"], k
            ref.step(1)
        m = L.lbm_read_monitor(sim.ctx, 0)
        last = L.lbm_monitor.from_address(buf.data_ptr() + (nsteps - 1) * size)
        assert m["time"] == last.time and m["sum_phi"] == last.sum_phi
        for a, b in zip(sim.populations(0), ref.populations(0)):
            assert np.array_equal(a, b)
