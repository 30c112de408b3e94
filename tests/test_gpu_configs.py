"""The full-size configurations run for their stated step counts: the batched
512-instance set for 5000 steps in every storage form against the GPU FP64 form
(itself tied to the oracle on sampled instances), the 512 x 512 spinodal for
20000 steps against the oracle's stored samples, and the 1024 x 4096 rising
bubble for 50000 steps in both variants (IM, QIM) and every form against FP64.

Error metric (field-max normalised) and the FP32 / FP16 bars as in
test_gpu_parity.py; measured values go to the parity report.
"""
import os

import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REDUCED = ("f32", "f32_c", "f32_cc", "f32_g16", "f32_h16")
CONSERVATIVE = ("f32_c", "f32_cc", "f32_g16", "f32_h16")


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
    den = np.max(np.hypot(b["ux"], b["uy"]))
    return float(np.max(np.hypot(a["ux"] - b["ux"], a["uy"] - b["uy"])) / (den if den > 0 else 1.0))


def test_batched_512_for_5000_steps(L, orc, report):
    # Configuration: 512 droplets / bubbles, N in {32..256}, 5000 steps, graph-captured.
    cfgs = wl.batched_mixed(512)
    phis = [wl.initial_phi(c) for c in cfgs]
    n = 5000

    def run(form):
        with L.Simulation(cfgs, form, phi0=phis) as sim:
            sim.step(n)
            return ([sim.fields(k, ("phi", "ux", "uy")) for k in range(len(cfgs))],
                    [sim.diagnostics(k) for k in range(len(cfgs))])

    # N = 32 bubbles at density ratio 100 (R = 8 = 2W) sit at the method's limit:
    # 6 of these 24 diverge in the FP64 oracle itself after 4000-5000 steps (IM as
    # well as QIM; the same bubble at N = 64 is stable), and reduced precision
    # can tip one or two more. They are reported apart; every other instance must
    # stay finite in every form and enters the accuracy statistics.
    fragile = {k for k, c in enumerate(cfgs) if c["nx"] == 32 and c["walls_y"] == 1 and c["rho_A"] == 100.0}
    runs = {"f64": run("f64")}
    # the FP64 form against the oracle on small instances (all 5000 steps)
    small = [k for k, c in enumerate(cfgs) if c["nx"] == 32 and k not in fragile][:6]
    for k in small:
        P = orc.params(cfgs[k])
        st = orc.init(P, phis[k])
        orc.step(P, st, n)
        ref = orc.fields(P, st)
        got = runs["f64"][0][k]
        assert rel(got["phi"], ref["phi"]) < 1e-10, k
        assert rel_u(got, ref) < 1e-10, k
    drops = [k for k, c in enumerate(cfgs) if c["walls_y"] == 0]
    keep = [k for k in range(len(cfgs)) if k not in fragile]
    f64_fields, f64_diag = runs["f64"]
    summary = {"f64": {"fragile_nonfinite": sorted(k for k in fragile if f64_diag[k]["status"] != L.LBM_OK)}}
    assert all(f64_diag[k]["status"] == L.LBM_OK for k in keep)
    for form in REDUCED:
        fields, diag = run(form)
        assert all(diag[k]["status"] == L.LBM_OK for k in keep), form
        e_phi = [rel(fields[k]["phi"], f64_fields[k]["phi"]) for k in keep]
        e_u = [rel_u(fields[k], f64_fields[k]) for k in keep]
        drift = [abs(diag[k]["sum_phi"] - phis[k].sum()) / phis[k].sum() for k in keep]
        dp = lambda d: d["P_bulk_A"] - d["P_bulk_B"]
        e_dp = [abs(dp(diag[k]) - dp(f64_diag[k])) / abs(dp(f64_diag[k])) for k in drops]
        summary[form] = {"phi_max": max(e_phi), "phi_median": float(np.median(e_phi)),
                         "u_max": max(e_u), "u_median": float(np.median(e_u)),
                         "mass_drift_max": max(drift), "laplace_dp_vs_f64_max": max(e_dp),
                         "laplace_dp_vs_f64_median": float(np.median(e_dp)),
                         "fragile_nonfinite": sorted(k for k in fragile if diag[k]["status"] != L.LBM_OK)}
    laplace_f64 = [abs(f64_diag[k]["P_bulk_A"] - f64_diag[k]["P_bulk_B"]) / wl.laplace_dp_expected(cfgs[k]) - 1
                   for k in drops]
    report(forms=summary, droplets=len(drops), fragile=len(fragile),
           f64_laplace_err_median=float(np.median(np.abs(laplace_f64))))
    # Mass: the conservative forms keep sum(phi) to 1e-6 (measured <= 8e-9).
    for form in CONSERVATIVE:
        assert summary[form]["mass_drift_max"] < 1e-6, (form, summary[form])
    # Fields and the Laplace jump against the FP64 form after 5000 steps. The
    # flow (bubbles rising, droplets relaxing) carries the reduced-precision
    # differences on: measured phi up to 4.2e-4 (FP32) / 1.0e-2 (FP16 g). The
    # jump of a droplet settles within ~1000 steps at an offset that then stays
    # (the FP32 arithmetic's quasi-equilibrium): median 2e-5 / 2e-4, worst single
    # droplet 1.5e-3 (two-float h_0) / 4e-2 (FP16), much the same with geometric
    # bulk masks as with the phi thresholds. Bars: 2.5x those.
    bars = {"f32": (1e-3, 0.2, 1e-3), "f32_c": (1e-3, 1e-2, 1e-4), "f32_cc": (1e-3, 1e-2, 1e-4),
            "f32_g16": (2.5e-2, 0.1, 5e-4), "f32_h16": (2.5e-2, 0.1, 5e-4)}
    for form, (b_phi, b_dp, b_dp_med) in bars.items():
        assert summary[form]["phi_max"] < b_phi, (form, summary[form])
        assert summary[form]["laplace_dp_vs_f64_max"] < b_dp, (form, summary[form])
        assert summary[form]["laplace_dp_vs_f64_median"] < b_dp_med, (form, summary[form])


def _spinodal_golden():
    blocks, cur = {}, None
    with open(os.path.join(GOLDEN, "spinodal_512_oracle_samples.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0] == "step":
                cur = int(t[1])
                blocks[cur] = {"max": None, "cells": []}
            elif t[0] == "max":
                blocks[cur]["max"] = [float(v) for v in t[1:]]
            else:
                blocks[cur]["cells"].append([int(t[0]), int(t[1])] + [float(v) for v in t[2:]])
    return blocks


def test_spinodal_512_for_20000_steps(L, report):
    # Configuration: 512 x 512 spinodal, QIM, 20000 steps; FP64 and the FP32 forms
    # against the oracle's samples at 2000 / 5000 / 10000 / 20000 steps.
    gold = _spinodal_golden()
    cfg = wl.spinodal()
    phi0 = wl.initial_phi(cfg)
    curve = {}
    for form in ("f64", "f32", "f32_c"):
        with L.Simulation(cfg, form, phi0=[phi0]) as sim:
            done = 0
            for n in sorted(gold):
                sim.step(n - done)
                done = n
                f = sim.fields(0, ("phi", "ux", "uy", "p"))
                cells = np.array(gold[n]["cells"])
                x, y = cells[:, 0].astype(int), cells[:, 1].astype(int)
                mx = gold[n]["max"]
                err = {}
                for j, name in enumerate(("phi", "ux", "uy", "p")):
                    err[name] = float(np.max(np.abs(f[name][y, x] - cells[:, 2 + j])) / mx[j])
                curve.setdefault(form, {})[n] = err
    report(curve=curve)
    for n, err in curve["f64"].items():
        assert max(err.values()) < 1e-10, (n, err)
    for form in ("f32", "f32_c"):
        assert curve[form][2000]["phi"] < 4 * 9 * 2.0 ** -24 * np.sqrt(2000), curve[form]
    # The two-float h_0 form stays at the FP32 rounding level through the linear
    # growth (7e-8 up to 10000 steps) and within 1e-3 once domains coarsen
    # (measured 7.7e-5 at 20000). Plain FP32 is reported only: its sum(phi) drifts
    # by up to 2^-24 a step, which shifts the mean composition the domains
    # coarsen around (phi 4.1e-2 off at 20000 steps).
    for n, err in curve["f32_c"].items():
        assert err["phi"] < 1e-3, (n, err)
        assert max(err["ux"], err["uy"]) < 2e-2, (n, err)


@pytest.mark.parametrize("qim", [1, 0])
def test_bubble_1024x4096_for_50000_steps(L, report, qim):
    # Configuration: rising bubble 1024 x 4096, 50000 steps; the FP64 form is the
    # long-run reference (its first steps are pinned to the oracle in
    # test_gpu_parity.py); every reduced form against it.
    cfg = wl.rising_bubble(qim=qim)
    phi0 = wl.initial_phi(cfg)
    n, every = 50000, 5000
    track = {}
    for form in ("f64",) + REDUCED:
        ys, drift = [], []
        with L.Simulation(cfg, form, phi0=[phi0]) as sim:
            y0 = sim.diagnostics(0)["centroid_B_y"]
            for t in range(every, n + 1, every):
                sim.step(every)
                d = sim.diagnostics(0)
                assert d["status"] == L.LBM_OK, (form, t)
                ys.append(d["centroid_B_y"] - y0)
                drift.append(abs(d["sum_phi"] - phi0.sum()) / phi0.sum())
        track[form] = (np.array(ys), drift)
    ref = track["f64"][0]
    rise = ref[-1]
    v_ref = (ref[-1] - ref[-3]) / (2 * every)
    out = {"rise_cells_f64": float(rise), "rise_velocity_f64": float(v_ref),
           "mass_drift_f64": track["f64"][1][-1]}
    for form in REDUCED:
        ys, drift = track[form]
        v = (ys[-1] - ys[-3]) / (2 * every)
        out[form] = {"centroid_vs_f64_over_rise": float(np.max(np.abs(ys - ref)) / rise),
                     "velocity_vs_f64": float(abs(v - v_ref) / abs(v_ref)),
                     "mass_drift": drift[-1]}
    report(**out)
    assert rise > 20.0                               # the bubble rises
    # Plain FP32 storage is reported, not held to a bar: phi ~ 1 sits in h_0 and
    # rounds the same way every step, so sum(phi) drifts by up to 2^-24 a step
    # (measured 3.5e-5 .. 7.9e-5 over 50000 steps) and the bubble's volume, hence
    # its buoyancy and rise, drift with it (centroid off by 4 - 13 % of the rise).
    # The conservative forms remove that drift.
    assert out["f32"]["mass_drift"] < n * 2.0 ** -24
    for form, bar in (("f32_c", 1e-3), ("f32_cc", 1e-3), ("f32_g16", 5e-2), ("f32_h16", 5e-2)):
        assert out[form]["centroid_vs_f64_over_rise"] < bar, (form, out[form])
        assert out[form]["velocity_vs_f64"] < 3 * bar, (form, out[form])
    for form in CONSERVATIVE:
        assert out[form]["mass_drift"] < 1e-8, (form, out[form])
