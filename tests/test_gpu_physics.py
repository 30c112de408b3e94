"""Long GPU runs of the paper's own validation settings (Sec. 4), compared with
the analytic solutions and, loosely, with the paper's printed accuracy.

These need 10^5 - 10^6 steps, out of reach of the CPU oracle in test time; the
GPU path they run is the one the parity tests pin to the oracle.
"""
import os

import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_08933_gb300 import build, lbm
    build.build()
    return lbm


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_laplace_table1_density_ratio_50(L, report):
    # Sec. 4.2, Table 1: 100 x 100 periodic, rho_A/rho_B = 50, tau_g = 0.8,
    # tau_h = 1, sigma = 0.001, M = 0.02, F_s = -phi grad(mu), W = 4, R = 20..40.
    table = _golden("table1_laplace_rho50.txt")
    cfgs = []
    for qim in (1, 0):
        for R in table[:, 0]:
            cfgs.append(wl.static_droplet(n=100, R=float(R), rho_ratio=50.0, sigma=0.001,
                                          tau_g=0.8, tau_h=1.0, M=0.02, qim=qim))
    with L.Simulation(cfgs, "f64", phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        sim.step(500000)
        errs = []
        for k, c in enumerate(cfgs):
            d = sim.diagnostics(k)
            assert d["status"] == L.LBM_OK
            errs.append(abs((d["P_bulk_A"] - d["P_bulk_B"]) / wl.laplace_dp_expected(c) - 1))
    n = len(table)
    qim_err, im_err = np.array(errs[:n]), np.array(errs[n:])
    report(qim_err_percent=list(100 * qim_err), im_err_percent=list(100 * im_err))
    # the paper reports at most 0.68 % (QIM) and 1.00 % (IM) at this setting
    assert np.all(qim_err < 0.02) and np.all(im_err < 0.02)


def test_layered_table2(L, report):
    # Sec. 4.3, Table 2: NY x NX = 100 x 10, walls in y, rho ratio 1, W = 4,
    # sigma = 0.001, M = 0.1, u_c = 5e-5, G = u_c (mu_A + mu_B) / h^2.
    table = _golden("table2_layered.txt")
    ny, nx, h = 100, 10, 50.0
    cfgs, drive = [], []
    for ratio in table[:, 0]:
        # the paper gives no relaxation times; the less viscous fluid takes
        # tau = 0.55 (reading Q15), so the other one's stays <= 50.5 at ratio 1000
        c = wl.layered_poiseuille(nx=nx, ny=ny, rho_ratio=1.0, mu_ratio=float(ratio), tau_min=0.55)
        muA, muB = c["rho_A"] * c["nu_A"], c["rho_B"] * c["nu_B"]
        c["force_x"] = 5e-5 * (muA + muB) / h ** 2
        cfgs.append(c)
        drive.append((muA, muB, c["force_x"]))
    errs = []
    with L.Simulation(cfgs, "f64", phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        prev = None
        for chunk in range(100):
            sim.step(20000)
            ux = np.stack([sim.fields(k, ("ux",))["ux"][:, 0] for k in range(len(cfgs))])
            if prev is not None and np.max(np.abs(ux - prev)) < 1e-9 * np.max(np.abs(ux)):
                break
            prev = ux
        yj = np.arange(ny) + 0.5 - ny / 2
        for k, (muA, muB, G) in enumerate(drive):
            # phase A below: the upper layer of Eq. 37 is fluid B
            muu, mud = muB, muA
            r = yj / h
            a = (muu - mud) / (muu + mud)
            ua = np.where(yj > 0, G * h * h / (2 * muu) * (-r * r - r * a + 2 * muu / (muu + mud)),
                          G * h * h / (2 * mud) * (-r * r - r * a + 2 * mud / (muu + mud)))
            errs.append(np.abs(ux[k] - ua).sum() / np.abs(ua).sum())
    report(err_percent=[100 * e for e in errs], paper_percent=list(table[:, 1]))
    # no worse than the paper's Table 2 at the same ratios
    assert np.all(np.array(errs) < table[:, 1] / 100)


def _sweep_golden():
    cases, cur = {}, None
    with open(os.path.join(GOLDEN, "layered_sweep_8x256_oracle.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if line.startswith("case"):
                _, rr, mr, steps, err = line.split()
                cur = (float(rr), float(mr))
                cases[cur] = {"steps": int(steps), "err": float(err), "ux": []}
            else:
                cases[cur]["ux"].extend(float(v) for v in line.split())
    return cases


@pytest.mark.parametrize("form", ["f64", "f32_c"])
def test_layered_sweep_8x256(L, report, form):
    # Configuration: 8 x 256 channel, A below, density ratio {1, 10, 100, 1000} x
    # dynamic viscosity ratio {1, 10, 100}, F_x = 1e-7, to steady state (at most
    # 4e6 steps). Compared with the FP64 oracle's steady profiles
    # (tests/golden/make_layered_sweep.py) and with Eq. 37. In FP32 storage the
    # slowest viscous mode stalls: late in the approach its change per step is
    # below one unit in the last place of the populations (u ~ 0.025, F = 1e-7),
    # so the low-viscosity cases stop short of the steady state; FP64 reaches it.
    gold = _sweep_golden()
    cfgs = []
    for rr in (1.0, 10.0, 100.0, 1000.0):
        for mr in (1.0, 10.0, 100.0):
            cfgs.append(wl.layered_poiseuille(rho_ratio=rr, mu_ratio=mr,
                                              viscosity=0 if rr == 1.0 else 1))
    ny, h = 256, 128.0
    with L.Simulation(cfgs, form, phi0=[wl.initial_phi(c) for c in cfgs]) as sim:
        prev, steps = None, 0
        for chunk in range(40):
            sim.step(100000)
            steps += 100000
            ux = np.stack([sim.fields(k, ("ux",))["ux"][:, 0] for k in range(len(cfgs))])
            if prev is not None and np.max(np.abs(ux - prev) / np.abs(ux).max(axis=1, keepdims=True)) < 2e-6:
                break
            prev = ux
        status = [sim.diagnostics(k)["status"] for k in range(len(cfgs))]
    yj = np.arange(ny) + 0.5 - ny / 2
    res = {}
    for k, c in enumerate(cfgs):
        rr, mr = c["rho_A"], c["rho_A"] * c["nu_A"] / (c["rho_B"] * c["nu_B"])
        muA, muB = c["rho_A"] * c["nu_A"], c["rho_B"] * c["nu_B"]
        G = c["force_x"]
        muu, mud = muB, muA
        r = yj / h
        a = (muu - mud) / (muu + mud)
        ua = np.where(yj > 0, G * h * h / (2 * muu) * (-r * r - r * a + 2 * muu / (muu + mud)),
                      G * h * h / (2 * mud) * (-r * r - r * a + 2 * mud / (muu + mud)))
        g = gold[(rr, round(mr))]
        uo = np.array(g["ux"])
        res["rho%g_mu%g" % (rr, round(mr))] = {
            "l1_vs_eq37": float(np.abs(ux[k] - ua).sum() / np.abs(ua).sum()),
            "oracle_l1_vs_eq37": g["err"],
            "vs_oracle": float(np.max(np.abs(ux[k] - uo)) / np.max(np.abs(uo))),
            "status": int(status[k])}
    report(cases=res, steps=steps)
    bar = 1e-4 if form == "f64" else 3e-2
    for key, r in res.items():
        assert r["status"] == L.LBM_OK, key
        # the GPU reaches the method's own steady state (field-max metric)
        assert r["vs_oracle"] < bar, (key, r)
        assert abs(r["l1_vs_eq37"] - r["oracle_l1_vs_eq37"]) < bar, (key, r)
        # and where the method itself is accurate (density ratio <= 10), Eq. 37
        if key.startswith(("rho1_", "rho10_")):
            assert r["l1_vs_eq37"] < 0.05, (key, r)
