"""The slab decomposition on one GPU: the slabs of a domain are instances of one
context (one batched launch a step for all of them), and their ghost rows are
refreshed through device buffers with lbm_pack_rows / lbm_unpack_rows -- the
same exchange code a run with one slab per GPU uses, minus the transport. The
slabs' own rows must equal the undivided grid bit for bit in every storage
form (the FP16 scales depend on the parameters only, so every slab has the
undivided grid's)."""
import numpy as np
import pytest

from paper_1902_08933_gb300 import slab
from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
STEPS = 23


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def _case(name):
    if name == "bubble":
        cfg = wl.rising_bubble(nx=128, ny=160, R=20.0, cy=50.0, W=4.0, Re=10.0)
    else:
        cfg = wl.static_droplet(n=96, R=24.0)
    rng = np.random.default_rng(9)
    phi0 = np.clip(wl.initial_phi(cfg) + 0.01 * rng.standard_normal((cfg["ny"], cfg["nx"])), 0, 1)
    return cfg, phi0


@pytest.mark.parametrize("form", ["f64", "f32", "f32_c", "f32_cc", "f32_g16", "f32_h16"])
@pytest.mark.parametrize("case,world,ghost", [("bubble", 2, 3), ("bubble", 4, 9), ("droplet", 3, 6)])
def test_slabs_in_one_context_equal_undivided(L, form, case, world, ghost):
    import torch
    cfg, phi0 = _case(case)
    periodic = not cfg["walls_y"]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        with L.Simulation(cfg, form, stream=stream.cuda_stream, phi0=[phi0]) as ref:
            ref.step(STEPS)
            rh, rg = ref.populations(0)
        slabs = slab.plan(cfg["ny"], world, ghost, periodic)
        cfgs = [slab.local_config(cfg, s, world) for s in slabs]
        phis = [slab.local_field(phi0, s) for s in slabs]
        with L.Simulation(cfgs, form, stream=stream.cuda_stream, phi0=phis) as sim:
            run = slab.SlabRun(slabs, ghost, {s.rank: slab.GpuSlab(L, sim, s.rank) for s in slabs}, periodic)
            run.start()
            run.advance(5)
            run.advance(STEPS - 5)
            for s in slabs:
                h, g = sim.populations(s.rank)
                assert np.array_equal(h[:, s.lo:s.lo + s.own], rh[:, s.y0:s.y1]), (form, case, s.rank)
                assert np.array_equal(g[:, s.lo:s.lo + s.own], rg[:, s.y0:s.y1]), (form, case, s.rank)


def test_row_exchange_arguments(L):
    import torch
    cfg, phi0 = _case("bubble")
    with L.Simulation(cfg, "f32_c", phi0=[phi0]) as sim:
        rb = L.lbm_row_bytes(sim.ctx, 0)
        # h_1..8 and g (FP32), the h_0 pair (8 bytes), phi u (2 x FP32), p (FP32)
        assert rb == cfg["nx"] * (8 * 4 + 8 + 9 * 4 + 2 * 4 + 4)
        assert L.lbm_row_bytes(sim.ctx, 1) == 0
        buf = torch.zeros(3 * rb, dtype=torch.uint8, device="cuda")
        L.lbm_pack_rows(sim.ctx, 0, 10, 3, buf.data_ptr(), buf.numel())
        for args in ((0, cfg["ny"] - 2, 3), (0, -1, 1), (0, 0, 0), (1, 0, 1)):
            with pytest.raises(L.LbmError):
                L.lbm_pack_rows(sim.ctx, *args, buf.data_ptr(), buf.numel())
        with pytest.raises(L.LbmError):
            L.lbm_unpack_rows(sim.ctx, 0, 0, 4, buf.data_ptr(), buf.numel())   # buffer too small
        # a pack / unpack round trip leaves the state as it was, bit for bit;
        # unpacking those rows elsewhere copies them there
        sim.step(3)
        h0, g0 = sim.populations(0)
        L.lbm_pack_rows(sim.ctx, 0, 10, 3, buf.data_ptr(), buf.numel())
        L.lbm_unpack_rows(sim.ctx, 0, 10, 3, buf.data_ptr(), buf.numel())
        h1, g1 = sim.populations(0)
        assert np.array_equal(h0, h1) and np.array_equal(g0, g1)
        L.lbm_unpack_rows(sim.ctx, 0, 40, 3, buf.data_ptr(), buf.numel())
        h2, g2 = sim.populations(0)
        assert np.array_equal(h2[:, 40:43], h0[:, 10:13]) and np.array_equal(g2[:, 40:43], g0[:, 10:13])
        assert np.array_equal(h2[:, :40], h0[:, :40]) and np.array_equal(h2[:, 43:], h0[:, 43:])
