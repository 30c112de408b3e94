"""Failure detection on the GPU without a fault: a bounded device wait that runs
out is reported through the status word, the CUDA context stays usable, and a
checkpoint restores a state that continues exactly as an undisturbed run."""
import time

import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def _bubble():
    return wl.rising_bubble(nx=48, ny=40, R=8.0, cy=14.0, Re=5.0)


@pytest.mark.parametrize("precision", ["f64", "f32_c"])
def test_wait_timeout_is_reported_and_checkpoint_recovers(L, tmp_path, precision):
    cfg = _bubble()
    ckpt = str(tmp_path / "state.bin")
    with L.Simulation([cfg], precision, phi0=[wl.initial_phi(cfg)]) as ref, \
            L.Simulation([cfg], precision, phi0=[wl.initial_phi(cfg)]) as sim, \
            L.Simulation([cfg], precision, phi0=[wl.initial_phi(cfg)]) as other:
        ref.step(30)
        expected = ref.fields(0)
        sim.step(10)
        L.lbm_save(sim.ctx, ckpt)
        sim.step(7)
        t0 = time.perf_counter()
        L.lbm_inject_wait_timeout(sim.ctx, 1 << 14)
        with pytest.raises(L.LbmError) as e:
            sim.sync()
        elapsed = time.perf_counter() - t0
        assert e.value.status == L.LBM_ETIMEOUT
        assert "bounded device wait" in L.lbm_last_error(sim.ctx)
        assert elapsed < 10.0
        # the status is sticky: every read of the suspect state reports it
        with pytest.raises(L.LbmError) as e:
            sim.fields(0, ("phi",))
        assert e.value.status == L.LBM_ETIMEOUT
        with pytest.raises(L.LbmError) as e:
            sim.diagnostics(0)
        assert e.value.status == L.LBM_ETIMEOUT
        # the CUDA context is intact: another context steps and reads normally
        other.step(5)
        assert other.diagnostics(0)["status"] == L.LBM_OK
        # restoring the checkpoint clears the status; the run continues exactly
        L.lbm_load(sim.ctx, ckpt)
        sim.step(20)
        got = sim.fields(0)
        for k in expected:
            np.testing.assert_array_equal(got[k], expected[k])


def test_wait_timeout_rounds_are_checked(L):
    cfg = _bubble()
    with L.Simulation([cfg], "f64", phi0=[wl.initial_phi(cfg)]) as sim:
        for bad in (0, -1, (1 << 21) + 1):
            with pytest.raises(L.LbmError) as e:
                L.lbm_inject_wait_timeout(sim.ctx, bad)
            assert e.value.status == L.LBM_EINVAL
        sim.step(2)
        sim.sync()


def test_batched_wait_timeout_is_reported_and_checkpoint_recovers(L, tmp_path):
    """The batched launch's own wait (an item of step s waits for its instance's
    step s - 1): made to run out, it is reported like any bounded wait, the launch
    stops handing out work, and the queue and counters are left ready for the
    next launch (the restored run continues exactly)."""
    cfgs = [wl.rising_bubble(nx=48, ny=40, R=8.0, cy=14.0, Re=5.0), wl.static_droplet(n=32, R=8.0),
            wl.static_droplet(n=64, R=12.0)]
    phis = [wl.initial_phi(c) for c in cfgs]
    ckpt = str(tmp_path / "batched.bin")
    with L.Simulation(cfgs, "f32_c", phi0=phis) as ref, L.Simulation(cfgs, "f32_c", phi0=phis) as sim:
        for s in (ref, sim):
            L.lbm_set_pipeline(s.ctx, L.LBM_PIPELINE_BATCHED)
        ref.step(30)
        expected = [ref.populations(k) for k in range(len(cfgs))]
        sim.step(10)
        L.lbm_save(sim.ctx, ckpt)
        sim.step(7)
        t0 = time.perf_counter()
        L.lbm_inject_batched_wait_timeout(sim.ctx, 1 << 12)
        with pytest.raises(L.LbmError) as e:
            sim.sync()
        assert e.value.status == L.LBM_ETIMEOUT
        assert time.perf_counter() - t0 < 10.0
        L.lbm_load(sim.ctx, ckpt)
        sim.step(20)
        for k in range(len(cfgs)):
            for a, b in zip(sim.populations(k), expected[k]):
                np.testing.assert_array_equal(a, b)


def test_batched_wait_timeout_needs_the_batched_plan(L):
    cfg = _bubble()
    with L.Simulation([cfg], "f32_c", phi0=[wl.initial_phi(cfg)]) as sim:
        with pytest.raises(L.LbmError) as e:
            L.lbm_inject_batched_wait_timeout(sim.ctx, 100)
        assert e.value.status == L.LBM_ESTATE
        L.lbm_set_pipeline(sim.ctx, L.LBM_PIPELINE_BATCHED)
        for bad in (0, (1 << 21) + 1):
            with pytest.raises(L.LbmError) as e:
                L.lbm_inject_batched_wait_timeout(sim.ctx, bad)
            assert e.value.status == L.LBM_EINVAL
        sim.step(3)
        sim.sync()
