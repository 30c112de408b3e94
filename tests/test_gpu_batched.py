"""The batched launch (LBM_PIPELINE_BATCHED, the default for several instances):
every instance of a context advanced by ONE persistent kernel launch a step, whose
blocks take descriptors from an on-device queue: one strip of up to 256 columns
on the whole block, or two strips of up to 128 columns on two thread groups.

It runs the same per-cell arithmetic as the per-class paired kernels
(LBM_PIPELINE_PAIRS, one launch per strip width), only split into other strips
and scheduled differently, so the populations must agree bit for bit; the
per-class kernels are held to the oracle in test_gpu_parity.py. Mixed grids:
one wide strip (160), a wide strip and a narrow ragged last one (300), exactly
one narrow strip (128), narrower (96, 64, 34), walls and periodic y, odd ny,
both march directions (runs of 5 rows).
"""
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


def mixed_set():
    cfgs = [wl.rising_bubble(nx=160, ny=41, R=9, cy=14, W=4.0, Re=5.0),
            wl.static_droplet(n=128, R=30),
            wl.rising_bubble(nx=300, ny=37, R=8, cy=13, W=4.0, Re=8.0),
            wl.static_droplet(n=96, R=20),
            wl.rising_bubble(nx=64, ny=50, R=10, cy=16, W=4.0, Re=5.0),
            wl.static_droplet(n=34, R=8)]
    rng = np.random.default_rng(11)
    phis = [np.clip(wl.initial_phi(c) + 0.01 * rng.standard_normal((c["ny"], c["nx"])), 0, 1)
            for c in cfgs]
    return cfgs, phis


def run(L, cfgs, phis, form, mode, rows, steps, graphs=True):
    with L.Simulation(cfgs, form, phi0=phis) as sim:
        L.lbm_set_pipeline(sim.ctx, mode)
        L.lbm_set_launch(sim.ctx, 0, rows)
        L.lbm_set_graphs(sim.ctx, graphs)
        infos = [L.lbm_launch_info(sim.ctx, i) for i in range(L.lbm_launches_per_step(sim.ctx))]
        for n in steps:
            sim.step(n)
        pops = [sim.populations(k) for k in range(len(cfgs))]
        diags = [sim.diagnostics(k) for k in range(len(cfgs))]
    return infos, pops, diags


@pytest.mark.parametrize("form", FORMS)
def test_batched_equals_per_class_pairs(L, form):
    cfgs, phis = mixed_set()
    steps = (1, 20, 3)       # odd start, a graph replay, a direct remainder
    bi, bpops, bdiag = run(L, cfgs, phis, form, L.LBM_PIPELINE_AUTO, 5, steps)
    assert len(bi) == 1 and bi[0]["variant"] == "batched", bi
    pi, ppops, _ = run(L, cfgs, phis, form, L.LBM_PIPELINE_PAIRS, 5, steps)
    assert all(i["variant"] == "pairs" for i in pi) and len(pi) > 1, pi
    for k, ((hb, gb), (hp, gp)) in enumerate(zip(bpops, ppops)):
        assert np.array_equal(hb, hp) and np.array_equal(gb, gp), (form, k)
        assert bdiag[k]["nonfinite"] == 0


@pytest.mark.parametrize("rows", [1, 8, 0])
def test_batched_run_lengths_and_graphs(L, rows):
    # one-row runs (every descriptor a prologue), 8-row runs, the planner's
    # choice; graph replays against direct launches
    cfgs, phis = mixed_set()
    _, a, _ = run(L, cfgs, phis, "f32_c", L.LBM_PIPELINE_BATCHED, rows, (2, 16, 1), graphs=True)
    _, b, _ = run(L, cfgs, phis, "f32_c", L.LBM_PIPELINE_BATCHED, rows, (2, 16, 1), graphs=False)
    _, c, _ = run(L, cfgs, phis, "f32_c", L.LBM_PIPELINE_PAIRS, 0, (2, 16, 1), graphs=False)
    for (ha, ga), (hb, gb), (hc, gc) in zip(a, b, c):
        assert np.array_equal(ha, hb) and np.array_equal(ga, gb)
        assert np.array_equal(ha, hc) and np.array_equal(ga, gc)


def test_batched_single_instance_and_fallback(L):
    # BATCHED on one instance runs the persistent kernel too; an odd-nx instance
    # cannot use the paired kernel, so the context falls back to per-class launches
    cfg = wl.rising_bubble(nx=256, ny=64, R=12, cy=20, W=4.0, Re=5.0)
    phi = wl.initial_phi(cfg)
    bi, (a,), _ = run(L, [cfg], [phi], "f32", L.LBM_PIPELINE_BATCHED, 0, (9,))
    assert bi[0]["variant"] == "batched"
    pi, (b,), _ = run(L, [cfg], [phi], "f32", L.LBM_PIPELINE_AUTO, 0, (9,))
    assert pi[0]["variant"] == "pairs"
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    odd = [cfg, wl.static_droplet(n=33, R=8)]
    infos, _, _ = run(L, odd, [phi, wl.initial_phi(odd[1])], "f32", L.LBM_PIPELINE_BATCHED, 0, (2,))
    assert "batched" not in [i["variant"] for i in infos]


def test_batched_monitor_matches_diagnostics(L):
    # the monitored step through the batched kernel: the last group of each
    # instance to finish writes that instance's record; it must match the FP64
    # diagnostics of the same time level within the bars of test_gpu_monitor.py
    # (phi is stored in FP32 per cell; u and rho in the kernel's FP32 arithmetic)
    cfgs, phis = mixed_set()
    with L.Simulation(cfgs, "f32_c", phi0=phis) as sim:
        assert L.lbm_launch_info(sim.ctx, 0)["variant"] == "batched"
        sim.step(7)
        ref = [sim.diagnostics(k) for k in range(len(cfgs))]
        L.lbm_set_monitor(sim.ctx, True)
        for rep in range(2):   # twice: the arrival counters must be back at zero
            sim.step(1)
            for k, c in enumerate(cfgs):
                m = L.lbm_read_monitor(sim.ctx, k)
                assert m["status"] == L.LBM_OK and m["time"] == 7 + rep
                if rep == 0:
                    cells = c["nx"] * c["ny"]
                    assert abs(m["sum_phi"] - ref[k]["sum_phi"]) <= cells * 2.0 ** -24
                    assert abs(m["kinetic_energy"] - ref[k]["kinetic_energy"]) <= 1e-4 * ref[k]["kinetic_energy"]
                    assert abs(m["max_u"] - ref[k]["max_u"]) <= 1e-4 * ref[k]["max_u"]


def test_batched_512_is_one_launch(L):
    cfgs = wl.batched_mixed(512)
    with L.Simulation(cfgs, "f32_g16", phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        assert L.lbm_launches_per_step(sim.ctx) == 1
        info = L.lbm_launch_info(sim.ctx, 0)
        assert info["variant"] == "batched" and info["tile_x"] == 128
        sim.step(10)
        assert all(sim.diagnostics(k)["nonfinite"] == 0 for k in (0, 100, 511))
