"""The per-step monitor fused into the step kernels: sum(phi), kinetic energy and
max |u| of the monitored step's input time level, against the FP64 oracle's
diagnostics of the same state, and against sums of the GPU's own fields."""
import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
FORMS = ["f64", "f32", "f32_c", "f32_cc", "f32_g16", "f32_h16"]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def _cases():
    return {"bubble": wl.rising_bubble(nx=48, ny=40, R=8.0, cy=14.0, Re=5.0),
            "droplet": wl.static_droplet(n=64, R=16.0)}


def _own_sums(f):
    uu = f["ux"] ** 2 + f["uy"] ** 2
    return f["phi"].sum(), (0.5 * f["rho"] * uu).sum(), np.sqrt(uu.max())


@pytest.mark.parametrize("pipeline", ["auto", "plain"])
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["bubble", "droplet"])
def test_monitor_matches_oracle_and_own_fields(L, orc, report, case, form, pipeline):
    cfg = _cases()[case]
    phi0 = wl.initial_phi(cfg)
    n = 40
    P = orc.params(cfg)
    st = orc.init(P, phi0)
    orc.step(P, st, n - 1)
    ref = orc.diagnostics(P, st)
    with L.Simulation(cfg, form, phi0=[phi0]) as sim, L.Simulation(cfg, form, phi0=[phi0]) as own:
        L.lbm_set_pipeline(sim.ctx, {"auto": 0, "plain": 1}[pipeline])
        L.lbm_set_pipeline(own.ctx, {"auto": 0, "plain": 1}[pipeline])
        L.lbm_set_monitor(sim.ctx, True)
        sim.step(n)
        m = L.lbm_read_monitor(sim.ctx, 0)
        own.step(n - 1)
        f = own.fields(0, ("phi", "ux", "uy", "rho"))
    assert m["status"] == L.LBM_OK and m["time"] == n - 1
    mass, ke, umax = _own_sums(f)
    e_mass = abs(m["sum_phi"] - ref["sum_phi"]) / ref["sum_phi"]
    e_ke = abs(m["kinetic_energy"] - ref["kinetic_energy"]) / ref["kinetic_energy"]
    e_u = abs(m["max_u"] - ref["max_u"]) / ref["max_u"]
    report(mass=e_mass, ke=e_ke, max_u=e_u)
    cells = cfg["nx"] * cfg["ny"]
    if form == "f64":
        assert e_mass < 1e-13 and e_ke < 1e-10 and e_u < 1e-10
        assert abs(m["sum_phi"] - mass) <= 1e-13 * mass
        assert abs(m["kinetic_energy"] - ke) <= 1e-12 * ke
        assert abs(m["max_u"] - umax) <= 1e-13 * umax
    else:
        # against the oracle: phi within the FP32 storage bar per cell, u within
        # the parity bar of the form (2e-2 FP32 storage, 0.1 FP16)
        # (the static droplet's velocity is spurious currents near the rounding
        # level, so its u is compared with the GPU's own fields only)
        bar_u = 2e-2 if form in ("f32", "f32_c") else 0.1
        assert abs(m["sum_phi"] - ref["sum_phi"]) <= cells * 4 * 9 * 2.0 ** -24 * np.sqrt(n)
        if case == "bubble":
            assert e_u < bar_u and e_ke < 2 * bar_u + bar_u ** 2
        # against the GPU's own fields: those round phi to FP32 per cell (at most
        # 2^-24 |phi| each); u and rho come from the same arithmetic up to FMA contraction
        assert abs(m["sum_phi"] - mass) <= cells * 2.0 ** -24
        assert abs(m["kinetic_energy"] - ke) <= 1e-4 * ke
        assert abs(m["max_u"] - umax) <= 1e-4 * umax


@pytest.mark.parametrize("form", FORMS)
def test_monitoring_does_not_change_the_state(L, form):
    cfg = _cases()["bubble"]
    phi0 = wl.initial_phi(cfg)
    with L.Simulation(cfg, form, phi0=[phi0]) as a, L.Simulation(cfg, form, phi0=[phi0]) as b:
        L.lbm_set_monitor(a.ctx, True)
        for _ in range(10):
            a.step(7)                      # graph replays plus a monitored last step
        b.step(70)
        fa, fb = a.fields(0), b.fields(0)
        ha, ga = a.populations(0)
        hb, gb = b.populations(0)
    for k in fa:
        np.testing.assert_array_equal(fa[k], fb[k])
    np.testing.assert_array_equal(ha, hb)
    np.testing.assert_array_equal(ga, gb)


def test_monitor_sees_phi_conserved_fp32_c(L, report):
    # the two-float h_0 form keeps sum(phi) to ~1e-11 over thousands of steps
    cfg = _cases()["droplet"]
    phi0 = wl.initial_phi(cfg)
    with L.Simulation(cfg, "f32_c", phi0=[phi0]) as sim:
        L.lbm_set_monitor(sim.ctx, True)
        sim.step(1)
        m0 = L.lbm_read_monitor(sim.ctx, 0)
        sim.step(4000)
        m1 = L.lbm_read_monitor(sim.ctx, 0)
    drift = abs(m1["sum_phi"] - m0["sum_phi"]) / m0["sum_phi"]
    report(drift=drift)
    assert m0["time"] == 0 and m1["time"] == 4000
    assert abs(m0["sum_phi"] - phi0.sum()) <= 1e-9 * phi0.sum()
    assert drift < 1e-9


def test_monitor_batched_matches_single_contexts(L):
    cfgs = [wl.static_droplet(n=32, R=8.0), wl.rising_bubble(nx=64, ny=48, R=10.0, cy=16.0, Re=5.0),
            wl.static_droplet(n=48, R=12.0, rho_ratio=2.0)]
    phis = [wl.initial_phi(c) for c in cfgs]
    with L.Simulation(cfgs, "f64", phi0=phis) as sim:
        L.lbm_set_monitor(sim.ctx, True)
        sim.step(25)
        got = [L.lbm_read_monitor(sim.ctx, k) for k in range(len(cfgs))]
    for k, c in enumerate(cfgs):
        with L.Simulation(c, "f64", phi0=[phis[k]]) as one:
            L.lbm_set_monitor(one.ctx, True)
            one.step(25)
            m = L.lbm_read_monitor(one.ctx, 0)
        assert got[k]["time"] == m["time"] == 24
        for q in ("sum_phi", "kinetic_energy", "max_u"):
            assert abs(got[k][q] - m[q]) <= 1e-13 * abs(m[q]), (k, q)


def test_monitor_states_and_nonfinite(L):
    cfg = wl.static_droplet(n=16)
    phi0 = wl.initial_phi(cfg)
    with L.Simulation(cfg, "f32_c", phi0=[phi0]) as sim:
        with pytest.raises(L.LbmError) as e:
            L.lbm_read_monitor(sim.ctx, 0)            # never enabled
        assert e.value.status == L.LBM_ESTATE
        L.lbm_set_monitor(sim.ctx, True)
        with pytest.raises(L.LbmError) as e:
            L.lbm_read_monitor(sim.ctx, 0)            # no monitored step yet
        assert e.value.status == L.LBM_ESTATE
        sim.step(3)
        assert L.lbm_read_monitor(sim.ctx, 0)["time"] == 2
        sim.init(0, phi0)
        with pytest.raises(L.LbmError) as e:
            L.lbm_read_monitor(sim.ctx, 0)            # the instance was re-initialised
        assert e.value.status == L.LBM_ESTATE
        bad = phi0.copy()
        bad[3, 4] = np.nan
        sim.init(0, bad)
        sim.step(1)
        m = L.lbm_read_monitor(sim.ctx, 0)
        assert m["status"] == L.LBM_ENONFINITE
        L.lbm_set_monitor(sim.ctx, False)
        sim.init(0, phi0)
        sim.step(2)
        with pytest.raises(L.LbmError) as e:
            L.lbm_read_monitor(sim.ctx, 0)            # monitor off: nothing recorded
        assert e.value.status == L.LBM_ESTATE


def _record(L, buf):
    import ctypes
    return L.lbm_monitor.from_address(buf.data_ptr())


def test_async_read_matches_and_times_are_per_instance(L):
    import torch
    cfgs = [wl.static_droplet(n=32, R=8.0), wl.static_droplet(n=40, R=10.0)]
    phis = [wl.initial_phi(c) for c in cfgs]
    stream = torch.cuda.Stream()
    bufs = [torch.zeros(40, dtype=torch.uint8).pin_memory() for _ in range(2)]
    with L.Simulation(cfgs, "f32_c", stream=stream.cuda_stream, phi0=phis) as sim:
        L.lbm_set_monitor(sim.ctx, True)
        sim.step(10)
        sim.init(1, phis[1])                  # instance 1 restarts at time 0
        sim.step(5)
        for k in range(2):
            L.lbm_read_monitor_async(sim.ctx, k, bufs[k].data_ptr())
        ev = torch.cuda.Event()
        ev.record(stream)
        sim.step(3)                           # a later monitored step: the copies stay intact
        ev.synchronize()
        recs = [_record(L, b) for b in bufs]
        assert (recs[0].time, recs[1].time) == (14, 4)
        assert recs[0].nonfinite == 0 and recs[0].device_status == 0
        sync0 = L.lbm_read_monitor(sim.ctx, 0)
        assert sync0["time"] == 17
    with L.Simulation(cfgs, "f32_c", stream=stream.cuda_stream, phi0=phis) as ref:
        L.lbm_set_monitor(ref.ctx, True)
        ref.step(15)
        m = L.lbm_read_monitor(ref.ctx, 0)
    assert m["time"] == 14
    assert (m["sum_phi"], m["kinetic_energy"], m["max_u"]) == (recs[0].sum_phi, recs[0].kinetic_energy, recs[0].max_u)


def test_monitor_record_carries_a_wait_timeout(L):
    cfg = wl.static_droplet(n=16)
    with L.Simulation(cfg, "f32_c", phi0=[wl.initial_phi(cfg)]) as sim:
        L.lbm_set_monitor(sim.ctx, True)
        L.lbm_inject_wait_timeout(sim.ctx, 1 << 12)
        sim.step(1)
        with pytest.raises(L.LbmError) as e:
            L.lbm_read_monitor(sim.ctx, 0)
        assert e.value.status == L.LBM_ETIMEOUT


def test_step_monitored_writes_records_to_host(L):
    # lbm_step_monitored: the monitored step's kernels write each instance's
    # record into pinned host memory themselves; the records equal the ones
    # lbm_read_monitor returns, call after call, batched launch included
    import ctypes
    import torch
    cfgs = [wl.rising_bubble(nx=96, ny=64, R=10.0, cy=20.0, Re=5.0), wl.static_droplet(n=64, R=16.0),
            wl.static_droplet(n=48, R=11.0)]
    n = len(cfgs)
    size = ctypes.sizeof(L.lbm_monitor)
    slots = [torch.zeros(n * size, dtype=torch.uint8).pin_memory() for _ in range(2)]
    with L.Simulation(cfgs, "f32_c", phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        L.lbm_set_monitor(sim.ctx, True)
        for call in range(4):
            slot = slots[call % 2]
            slot.zero_()
            L.lbm_step_monitored(sim.ctx, 3, slot.data_ptr())
            sim.sync()
            for k in range(n):
                r = L.lbm_monitor.from_address(slot.data_ptr() + k * size)
                m = L.lbm_read_monitor(sim.ctx, k)
                assert r.time == 3 * call + 2 == m["time"]
                assert r.nonfinite == 0 and r.device_status == 0
                assert (r.sum_phi, r.kinetic_energy, r.max_u) == (m["sum_phi"], m["kinetic_energy"], m["max_u"])
        with pytest.raises(L.LbmError):
            L.lbm_step_monitored(sim.ctx, 0, slots[0].data_ptr())
        L.lbm_set_monitor(sim.ctx, False)
        with pytest.raises(L.LbmError):
            L.lbm_step_monitored(sim.ctx, 1, slots[0].data_ptr())
