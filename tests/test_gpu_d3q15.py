"""GPU D3Q15 path versus the FP64 D3Q15 oracle, element by element on seeded inputs.

Same metric and bars as the D2Q9 parity tests (test_gpu_parity.py): FP64 within
1e-12 on tiny grids over every flag combination and 1e-10 on larger grids;
FP32 storage within the per-cell rounding bar for phi and 2e-2 of the field
maximum for u and p.
"""
import itertools

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


def rel(a, b):
    den = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / (den if den > 0 else 1.0))


def rel_u(a, b):
    du = np.sqrt((a["ux"] - b["ux"]) ** 2 + (a["uy"] - b["uy"]) ** 2 + (a["uz"] - b["uz"]) ** 2)
    den = np.max(np.sqrt(b["ux"] ** 2 + b["uy"] ** 2 + b["uz"] ** 2))
    return float(np.max(du) / (den if den > 0 else 1.0))


def tol32_phi(n):
    return 4 * 15 * 2.0 ** -24 * np.sqrt(n)


def oracle_run(orc, cfg, phi0, n):
    P = orc.params(cfg)
    st = orc.init3(P, phi0)
    if n:
        orc.step3(P, st, n)
    return orc.fields3(P, st), st


def noisy(cfg, seed, amp=0.02):
    phi = wl.initial_phi(cfg)
    u = wl.uniform01(seed, phi.size).reshape(phi.shape)
    return np.clip(phi + amp * (2 * u - 1), -0.05, 1.05)


def compare(sim, k, ref, st, tol, fields=("phi", "ux", "uy", "uz", "p", "rho", "mu", "P"), pops=True):
    got = sim.fields(k)
    errs = {f: rel(got[f], ref[f]) for f in fields}
    if pops:
        h, g = sim.populations(k)
        errs["h"] = rel(h, st["h"])
        errs["g"] = rel(g, st["g"])
    bad = {f: e for f, e in errs.items() if not e <= tol}
    assert not bad, bad
    return errs


@pytest.mark.parametrize("walls,qim,pressure,sforce,visc",
                         list(itertools.product([0, 1], [0, 1], [0, 1, 2], [0, 1], [0, 1])))
def test_tiny_grids_all_flags_fp64(L, orc, walls, qim, pressure, sforce, visc):
    cfg = wl.static_droplet3(6, R=2.0)
    cfg.update(nx=7, ny=6, nz=5, walls_y=walls, qim=qim, pressure=pressure, surface_force=sforce,
               viscosity=visc, nu_B=0.05, gravity=1e-4 if walls else 0.0, force_x=1e-5)
    cfg["init"] = dict(kind="droplet", cx=3.5, cy=3.0, cz=2.5, R=2.0)
    phi0 = noisy(cfg, 11 + walls + 2 * qim + 4 * pressure + 12 * sforce + 24 * visc)
    ref, st = oracle_run(orc, cfg, phi0, 8)
    # FP64 runs the unfused step by default (AUTO) and the fused march under ASYNC
    for mode in (L.LBM_PIPELINE_AUTO, L.LBM_PIPELINE_ASYNC):
        with L.Simulation(cfg, "f64", phi0=[phi0]) as sim:
            L.lbm_set_pipeline(sim.ctx, mode)
            sim.step(8)
            compare(sim, 0, ref, st, 1e-12)


def test_initial_state_matches_oracle(L, orc):
    cfg = wl.rising_bubble3(nx=12, ny=10, nz=8, R=3.0, cy=4.0, Re=5.0)
    phi0 = noisy(cfg, 3)
    ref, st = oracle_run(orc, cfg, phi0, 0)
    for form, tol in (("f64", 1e-15), ("f32", 1e-6), ("f32_c", 1e-6)):
        with L.Simulation(cfg, form, phi0=[phi0]) as sim:
            h, g = sim.populations(0)
            assert rel(h, st["h"]) < tol and np.abs(g).max() == 0.0, form


def test_droplet_32_cubed(L, orc, report):
    cfg = wl.static_droplet3(32, R=9.0)
    phi0 = wl.initial_phi(cfg)
    n = 200
    ref, st = oracle_run(orc, cfg, phi0, n)
    with L.Simulation(cfg, "f64", phi0=[phi0]) as sim:
        sim.step(n)
        errs = compare(sim, 0, ref, st, 1e-10)
        report(**{"f64_" + k: v for k, v in errs.items()})
    for form in ("f32", "f32_c"):
        with L.Simulation(cfg, form, phi0=[phi0]) as sim:
            sim.step(n)
            got = sim.fields(0)
            e = {"phi": rel(got["phi"], ref["phi"]), "u": rel_u(got, ref), "p": rel(got["p"], ref["p"])}
            report(**{form + "_" + k: v for k, v in e.items()})
            assert e["phi"] < tol32_phi(n) and e["u"] < 2e-2 and e["p"] < 2e-2, (form, e)


@pytest.mark.parametrize("nx", [21, 22])
def test_bubble_with_walls_ragged(L, orc, report, nx):
    # walls normal to y, buoyancy, odd sizes
    cfg = wl.rising_bubble3(nx=nx, ny=26, nz=13, R=5.0, cy=9.0, Re=5.0)
    phi0 = wl.initial_phi(cfg)
    n = 100
    ref, st = oracle_run(orc, cfg, phi0, n)
    with L.Simulation(cfg, "f64", phi0=[phi0]) as sim:
        sim.step(n)
        compare(sim, 0, ref, st, 1e-10)
    for form in ("f32", "f32_c"):
        with L.Simulation(cfg, form, phi0=[phi0]) as sim:
            sim.step(n)
            got = sim.fields(0)
            e = {"phi": rel(got["phi"], ref["phi"]), "u": rel_u(got, ref), "p": rel(got["p"], ref["p"])}
            report(**{form + "_" + k: v for k, v in e.items()})
            assert e["phi"] < tol32_phi(n) and e["u"] < 2e-2 and e["p"] < 2e-2, (form, e)


def test_several_instances_in_one_context(L, orc):
    cfgs = [wl.static_droplet3(10, R=3.0), wl.rising_bubble3(nx=9, ny=12, nz=7, R=3.0, cy=4.5, Re=5.0),
            wl.static_droplet3(8, R=2.5, rho_ratio=2.0, qim=0)]
    phis = [noisy(c, 40 + k) for k, c in enumerate(cfgs)]
    refs = [oracle_run(orc, c, phis[k], 24) for k, c in enumerate(cfgs)]
    # the fused march (ASYNC): one launch for all instances; the default FP64
    # step (AUTO): the three unfused kernels an instance
    for mode, launches in ((L.LBM_PIPELINE_ASYNC, 1), (L.LBM_PIPELINE_AUTO, 3 * len(cfgs))):
        with L.Simulation(cfgs, "f64", phi0=phis) as sim:
            L.lbm_set_pipeline(sim.ctx, mode)
            sim.step(1)
            sim.step(23)        # graph replays from here on
            for k, c in enumerate(cfgs):
                compare(sim, k, refs[k][0], refs[k][1], 1e-12)
            assert L.lbm_launches_per_step(sim.ctx) == launches


def test_diagnostics_match_oracle(L, orc):
    cfg = wl.rising_bubble3(nx=16, ny=20, nz=12, R=4.0, cy=7.0, Re=5.0)
    phi0 = wl.initial_phi(cfg)
    _, st = oracle_run(orc, cfg, phi0, 30)
    od = orc.diagnostics3(orc.params(cfg), st)
    with L.Simulation(cfg, "f64", phi0=[phi0]) as sim:
        sim.step(30)
        d = sim.diagnostics(0)
    assert d["status"] == L.LBM_OK
    for k in ("sum_phi", "sum_rho", "kinetic_energy", "max_u", "centroid_B_x", "centroid_B_y",
              "P_bulk_A", "P_bulk_B"):
        assert abs(d[k] - od[k]) <= 1e-11 * max(abs(od[k]), 1e-300), k
    assert d["n_bulk_A"] == od["n_bulk_A"] and d["n_bulk_B"] == od["n_bulk_B"]


@pytest.mark.parametrize("form", ["f64", "f32", "f32_c"])
def test_phi_conserved_3d(L, report, form):
    cfg = wl.rising_bubble3(nx=32, ny=48, nz=24, R=7.0, cy=14.0, Re=10.0)
    phi0 = wl.initial_phi(cfg)
    n = 500
    with L.Simulation(cfg, form, phi0=[phi0]) as sim:
        sim.step(n)
        d = sim.diagnostics(0)
    drift = abs(d["sum_phi"] - phi0.sum()) / phi0.sum()
    report(drift=drift)
    assert d["status"] == L.LBM_OK
    assert drift < {"f64": 1e-13, "f32": n * 2.0 ** -24, "f32_c": 1e-9}[form], drift


def test_checkpoint_and_graphs_are_bitwise(L, tmp_path):
    cfg = wl.static_droplet3(12, R=3.5)
    phi0 = noisy(cfg, 9)
    path = str(tmp_path / "ck3.bin")
    with L.Simulation(cfg, "f32_c", phi0=[phi0]) as a:
        a.step(7)
        L.lbm_save(a.ctx, path)
        a.step(40)
        ha, ga = a.populations(0)
    with L.Simulation(cfg, "f32_c") as b:
        L.lbm_load(b.ctx, path)
        L.lbm_set_graphs(b.ctx, False)
        for _ in range(40):
            b.step(1)
        hb, gb = b.populations(0)
    assert np.array_equal(ha, hb) and np.array_equal(ga, gb)


def test_d3q15_context_rules(L):
    c2 = wl.static_droplet(16)
    c3 = wl.static_droplet3(8, R=2.0)
    with pytest.raises(L.LbmError):
        L.Simulation([c2, c3], "f64")                   # one lattice a context
    for form in ("f32_g16", "f32_h16", "f32_cc"):
        with pytest.raises(L.LbmError):
            L.Simulation([c3], form)                    # FP16 storage and compensated mu: D2Q9 only
    with L.Simulation([c3], "f64", phi0=[wl.initial_phi(c3)]) as sim:
        with pytest.raises(L.LbmError):
            L.lbm_set_monitor(sim.ctx, True)
        with pytest.raises(L.LbmError):
            L.lbm_launch_info(sim.ctx, 0)
        f = sim.fields(0, ("uz",))
        assert f["uz"].shape == (8, 8, 8)
    with L.Simulation([c2], "f64", phi0=[wl.initial_phi(c2)]) as sim:
        with pytest.raises(L.LbmError):
            sim.fields(0, ("uz",))                      # no uz on D2Q9


def test_laplace_law_sphere_gpu(L, report):
    # Sec. 4.2 in 3-D: Delta p = 2 sigma / R, 64^3 periodic, density ratio 10
    cfgs = [wl.static_droplet3(64, R=R) for R in (12.0, 16.0)]
    with L.Simulation(cfgs, "f64", phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        sim.step(10000)
        errs = []
        for k, c in enumerate(cfgs):
            d = sim.diagnostics(k)
            errs.append((d["P_bulk_A"] - d["P_bulk_B"]) / wl.laplace_dp_expected3(c) - 1)
    report(laplace_err=errs)
    assert all(abs(e) < 0.03 for e in errs), errs


@pytest.mark.parametrize("form", ["f64", "f32", "f32_c"])
def test_fused_march_equals_unfused_step(L, form):
    # the fused z-march (tiles of 32 x 8 columns, rings in shared memory) and the
    # three-kernel step do the same arithmetic: ragged tiles, walls, both march
    # directions, several instances in one launch
    cfgs = [wl.rising_bubble3(nx=45, ny=21, nz=17, R=5.0, cy=8.0, Re=5.0),
            wl.static_droplet3(12, R=3.5), wl.rising_bubble3(nx=34, ny=9, nz=30, R=3.0, cy=4.0, Re=5.0)]
    phis = [noisy(c, 70 + k) for k, c in enumerate(cfgs)]
    # (FP64: to round-off; FP32: the compiler may contract a product into an FMA in
    # one kernel and not in the other, so the FP32 bars of the parity tests apply)
    out = []
    for mode in (L.LBM_PIPELINE_ASYNC, L.LBM_PIPELINE_PLAIN):   # fused, unfused
        with L.Simulation(cfgs, form, phi0=phis) as sim:
            L.lbm_set_pipeline(sim.ctx, mode)
            for rows in (0, 3):
                L.lbm_set_launch(sim.ctx, 0, rows)
                sim.step(9)
            out.append([(sim.populations(k), sim.fields(k)) for k in range(len(cfgs))])
    for ((ha, ga), fa), ((hb, gb), fb) in zip(out[0], out[1]):
        if form == "f64":
            assert rel(ha, hb) <= 1e-13 and rel(ga, gb) <= 1e-12, (rel(ha, hb), rel(ga, gb))
        else:
            assert rel(fa["phi"], fb["phi"]) < tol32_phi(18)
            assert rel_u(fa, fb) < 2e-2 and rel(fa["p"], fb["p"]) < 2e-2

