"""Pins of the D3Q15 oracle (the model of Sec. 3 on the 3-D lattice of Sec. 2.2).

The same identities as the D2Q9 pins with d = 3: lattice isotropy, the moment
conditions of the equilibria and of the force distribution (App. A), the
printed-versus-literal G_0 relation, pressure recovery, stencil Fourier symbols
(Eq. 30), conservation, symmetry, and two physical checks -- Laplace's law for a
sphere (Delta p = 2 sigma / R) and the layered Poiseuille profile of Eq. 37.
"""
import numpy as np
import pytest

from paper_1902_08933_gb300 import workloads as wl

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(315)


def lat(orc):
    c, w, op = orc.lattice3()
    return c.T.astype(float), w, op


def test_d3q15_isotropy(orc):
    c, w, op = lat(orc)
    assert c.shape == (15, 3)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), CS2 * np.eye(3), atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-15)
    d = np.eye(3)
    expect = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                         + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), expect, atol=1e-15)
    for i in range(15):
        assert np.array_equal(c[op[i]], -c[i])
    assert np.array_equal(c[0], [0, 0, 0])
    assert all(np.abs(c[i]).sum() == 1 for i in range(1, 7))
    assert all(np.abs(c[i]).sum() == 3 for i in range(7, 15))
    assert np.isclose(w[0], 2 / 9) and np.allclose(w[1:7], 1 / 9) and np.allclose(w[7:], 1 / 72)


@pytest.mark.parametrize("rho0", [0.0, 1.0])
def test_geq3_moments(orc, rho0):
    c, w, _ = lat(orc)
    for _ in range(5):
        p, rho = RNG.uniform(-0.01, 0.01), RNG.uniform(0.5, 10)
        u = RNG.uniform(-0.05, 0.05, 3)
        g = orc.geq3(p, rho, u, rho0)
        assert np.isclose(g.sum(), rho0, atol=1e-14)                                  # M0
        assert np.allclose(g @ c, rho * u, atol=1e-15)                                # M1
        M2 = np.einsum("i,ia,ib->ab", g, c, c)
        assert np.allclose(M2, p * np.eye(3) + rho * np.outer(u, u), atol=1e-14)      # M2


def test_heq3_moments(orc):
    c, w, _ = lat(orc)
    for _ in range(5):
        phi, mu, eta = RNG.uniform(0, 1), RNG.uniform(-0.01, 0.01), RNG.uniform(0.1, 2)
        u = RNG.uniform(-0.05, 0.05, 3)
        h = orc.heq3(phi, mu, eta, u)
        assert np.isclose(h.sum(), phi, atol=1e-15)
        assert np.allclose(h @ c, phi * u, atol=1e-15)
        assert np.allclose(np.einsum("i,ia,ib->ab", h, c, c), eta * mu * CS2 * np.eye(3), atol=1e-15)


def test_force_distribution3_moments(orc):
    c, w, _ = lat(orc)
    for _ in range(5):
        rho, S1 = RNG.uniform(0.5, 10), RNG.uniform(-1e-3, 1e-3)
        u, F, Ft = RNG.uniform(-0.05, 0.05, 3), RNG.uniform(-1e-3, 1e-3, 3), RNG.uniform(-1e-3, 1e-3, 3)
        S = RNG.uniform(-1e-3, 1e-3)
        G = orc.force_dist3(S, rho, S1, F, Ft, u)
        assert np.isclose(G.sum(), S, atol=1e-16)
        assert np.allclose(G @ c, F, atol=1e-16)
        M2 = np.einsum("i,ia,ib->ab", G, c, c)
        expect = CS2 * S * np.eye(3) + np.outer(u, Ft) + np.outer(Ft, u) + (2 / 3) * rho * CS2 * S1 * np.eye(3)
        assert np.allclose(M2, expect, atol=1e-16)


def test_printed_G0_3d_differs_by_two_thirds_rho_S1(orc):
    # printed G_0 - Eq. 34 at i = 0 = omega_0 (1 - 1/d) rho S1 with d = 3
    for _ in range(5):
        rho, S1 = RNG.uniform(0.5, 10), RNG.uniform(-1e-3, 1e-3)
        u, F, dp = RNG.uniform(-0.05, 0.05, 3), RNG.uniform(-1e-3, 1e-3, 3), RNG.uniform(-1e-3, 1e-3, 3)
        drho = RNG.uniform(-1e-2, 1e-2, 3)
        S = u @ drho + rho * S1
        Ft = F - dp + CS2 * drho
        literal = orc.force_dist3(S, rho, S1, F, Ft, u)[0]
        printed = orc.G0_printed3(rho, S1, F, dp, u)
        assert np.isclose(printed - literal, (2 / 9) * (2 / 3) * rho * S1, rtol=0, atol=1e-16)


def test_source_R3_moments(orc):
    c, w, _ = lat(orc)
    tau_h = 0.8
    d = RNG.uniform(-1e-3, 1e-3, 3)
    R = orc.source_R3(tau_h, d)
    assert np.isclose(R.sum(), 0.0, atol=1e-17)
    assert np.allclose(R @ c, (1 - 1 / (2 * tau_h)) * d, atol=1e-17)


def test_pressure3_recovers_p(orc):
    # g = g^eq(p, u) with rho_0 = 0: Eq. 29 gives p + c_s^2/(1 - omega_0) S/2 = p + (3/14) S
    # and Eq. 28 adds c_s^2/(1 - omega_0) (tau_g - 1/2) G_0 = (3/7)(tau_g - 1/2) G_0.
    for _ in range(5):
        p, rho, S, G0, tau = RNG.uniform(-1e-2, 1e-2), RNG.uniform(1, 5), RNG.uniform(-1e-3, 1e-3), \
            RNG.uniform(-1e-3, 1e-3), RNG.uniform(0.6, 1.5)
        u = RNG.uniform(-0.05, 0.05, 3)
        g = orc.geq3(p, rho, u, 0.0)
        assert np.isclose(orc.pressure3(2, g, S, rho, u, tau, G0), p + 3 / 14 * S, atol=1e-15)
        assert np.isclose(orc.pressure3(0, g, S, rho, u, tau, G0), p + 3 / 14 * S + 3 / 7 * (tau - 0.5) * G0,
                          atol=1e-15)


def _p3(nx, ny, nz, walls=0):
    return dict(nx=nx, ny=ny, nz=nz, walls_y=walls, rho_A=10, rho_B=1, nu_A=0.1, nu_B=0.1, sigma=0.01, W=4,
                tau_h=0.8, M=0.02)


def test_stencil3_fourier_symbols(orc):
    c, w, _ = lat(orc)
    nx, ny, nz = 8, 6, 10
    P = orc.params(_p3(nx, ny, nz))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for k in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 2, 3), (3, 1, 2)]:
        kv = 2 * np.pi * np.array([k[0] / nx, k[1] / ny, k[2] / nz])
        ph = kv[0] * x + kv[1] * y + kv[2] * z
        f = np.cos(ph)
        lam = 6 * np.sum(w * (np.cos(c @ kv) - 1))                       # Eq. 30b symbol
        assert np.allclose(orc.lap3(P, f), lam * f, atol=1e-13)
        gx, gy, gz = orc.grad3(P, f)
        sym = 3 * np.einsum("i,ia->a", w * np.sin(c @ kv), c)             # Eq. 30a: i * sym
        for a, ga in enumerate((gx, gy, gz)):
            assert np.allclose(ga, -sym[a] * np.sin(ph), atol=1e-13)


def test_stream3_periodic_and_bounce_back(orc):
    nx, ny, nz = 5, 4, 3
    c, w, op = lat(orc)
    post = RNG.uniform(size=(15, nz, ny, nx))
    P = orc.params(_p3(nx, ny, nz, walls=0))
    pre = orc.stream3(P, post)
    for i in range(15):
        assert np.array_equal(pre[i], np.roll(post[i], shift=(int(c[i, 2]), int(c[i, 1]), int(c[i, 0])),
                                              axis=(0, 1, 2)))
    Pw = orc.params(_p3(nx, ny, nz, walls=1))
    prew = orc.stream3(Pw, post)
    for i in range(15):
        cy = int(c[i, 1])
        rolled = np.roll(post[i], shift=(int(c[i, 2]), cy, int(c[i, 0])), axis=(0, 1, 2))
        if cy == 0:
            assert np.array_equal(prew[i], rolled)
        else:
            yin = slice(1, ny) if cy > 0 else slice(0, ny - 1)
            assert np.array_equal(prew[i][:, yin], rolled[:, yin])
            yb = 0 if cy > 0 else ny - 1              # the row next to the wall it left
            assert np.array_equal(prew[i][:, yb], post[op[i]][:, yb])


def _run3(orc, cfg, n, phi0=None):
    P = orc.params(cfg)
    st = orc.init3(P, wl.initial_phi(cfg) if phi0 is None else phi0)
    orc.step3(P, st, n)
    return P, st


@pytest.mark.parametrize("walls", [0, 1])
def test_phi_conserved_3d(orc, walls):
    cfg = wl.rising_bubble3(nx=12, ny=14, nz=10, R=3.5, cy=6.0, Re=5.0) if walls else wl.static_droplet3(12, R=3.5)
    phi0 = wl.initial_phi(cfg)
    P, st = _run3(orc, cfg, 40)
    d = orc.diagnostics3(P, st)
    assert d["nonfinite"] == 0
    assert abs(d["sum_phi"] - phi0.sum()) < 1e-12 * phi0.sum()


def test_uniform_state_is_fixed_point_3d(orc):
    cfg = wl.static_droplet3(8, R=2.0)
    cfg["init"] = dict(kind="uniform", value=0.3)
    P, st = _run3(orc, cfg, 10)
    f = orc.fields3(P, st)
    assert np.allclose(f["phi"], 0.3, atol=1e-14, rtol=0)
    assert np.abs(np.stack([f["ux"], f["uy"], f["uz"]])).max() < 1e-14


def test_translation_equivariance_3d(orc):
    cfg = wl.static_droplet3(10, R=3.0)
    cfg["init"] = dict(kind="noise", seed=5, mean=0.5, amp=0.05)
    phi0 = wl.initial_phi(cfg)
    P, a = _run3(orc, cfg, 6, phi0)
    _, b = _run3(orc, cfg, 6, np.roll(phi0, (2, 3, 1), axis=(0, 1, 2)))
    assert np.array_equal(np.roll(a["h"], (2, 3, 1), axis=(1, 2, 3)), b["h"])
    assert np.array_equal(np.roll(a["g"], (2, 3, 1), axis=(1, 2, 3)), b["g"])


def test_im_equals_qim_at_equal_densities_3d(orc):
    cfg = wl.static_droplet3(10, R=3.0, rho_ratio=1.0)
    cfg["init"] = dict(kind="noise", seed=6, mean=0.5, amp=0.05)
    cq, ci = dict(cfg, qim=1), dict(cfg, qim=0)
    _, a = _run3(orc, cq, 5)
    _, b = _run3(orc, ci, 5)
    assert np.array_equal(a["h"], b["h"]) and np.array_equal(a["g"], b["g"])


def test_laplace_law_sphere(orc):
    # Sec. 4.2 in 3-D: Delta p = 2 sigma / R for a sphere of phase A (rho ratio 10).
    cfg = wl.static_droplet3(32, R=9.0)
    P, st = _run3(orc, cfg, 1500)
    d = orc.diagnostics3(P, st)
    dp = d["P_bulk_A"] - d["P_bulk_B"]
    assert abs(dp / wl.laplace_dp_expected3(cfg) - 1) < 0.05


def test_layered_poiseuille_3d_within_paper_table2(orc):
    # Sec. 4.3 (Eq. 37) on the 3-D lattice, mu_A / mu_B = 3, 100-row channel two
    # cells wide in x and z; Table 2 reports 1.04 % for this ratio in 2-D.
    ny, h = 100, 50.0
    cfg = wl.layered_poiseuille3(nx=2, ny=ny, nz=2, rho_ratio=1.0, mu_ratio=3.0, tau_min=1.0)
    muA, muB = cfg["rho_A"] * cfg["nu_A"], cfg["rho_B"] * cfg["nu_B"]
    G = 5e-5 * (muA + muB) / h ** 2
    cfg["force_x"] = G
    P = orc.params(cfg)
    st = orc.init3(P, wl.initial_phi(cfg))
    prev = None
    for _ in range(40):
        orc.step3(P, st, 2500)
        ux = orc.fields3(P, st)["ux"][0, :, 0].copy()
        if prev is not None and np.max(np.abs(ux - prev)) < 5e-7 * np.max(np.abs(ux)):
            break
        prev = ux
    yj = np.arange(ny) + 0.5 - ny / 2
    ua = np.array([orc.layered_ux(y, h, G, muB, muA) for y in yj])
    err = np.abs(ux - ua).sum() / np.abs(ua).sum()
    assert err < 0.0104, err


def test_laplace_law_sphere_with_mu_grad_phi_force(orc):
    # F_s = mu grad(phi) (Sec. 3.1) differs from -phi grad(mu) by grad(phi mu), so
    # Laplace's law holds for P with p replaced by p - phi mu; left as p the jump
    # is near twice 2 sigma / R (mu is about 2 sigma / R in both bulks).
    cfg = wl.static_droplet3(32, R=9.0)
    cfg["surface_force"] = 0
    P, st = _run3(orc, cfg, 1000)
    f = orc.fields3(P, st)
    bulk_A, bulk_B = f["phi"] > 1 - 1e-3, f["phi"] < 1e-3
    Pc = f["P"] - f["phi"] * f["mu"]
    expected = wl.laplace_dp_expected3(cfg)
    assert abs((Pc[bulk_A].mean() - Pc[bulk_B].mean()) / expected - 1) < 0.05
    assert abs((f["P"][bulk_A].mean() - f["P"][bulk_B].mean()) / expected - 2) < 0.25


@pytest.mark.parametrize("phase", [0.0, 1.0], ids=["phase-B", "phase-A"])
def test_hydrostatic_rest_under_buoyancy_3d(orc, phase):
    # Sec. 4.4 buoyancy -(rho - rho_A) g along -y: a uniform phase at rest between
    # walls keeps u = 0 with dp/dy = (rho_A - rho) g exactly (linear p).
    g = 1e-5
    cfg = wl.layered_poiseuille3(nx=2, ny=16, nz=2, force_x=0.0, rho_ratio=10.0)
    cfg.update(nu_A=1.0 / 6.0, nu_B=1.0 / 6.0, gravity=g, init=dict(kind="uniform", value=phase))
    P, st = _run3(orc, cfg, 10000)
    f = orc.fields3(P, st)
    expected = (cfg["rho_A"] - cfg["rho_B"]) * g if phase == 0.0 else 0.0
    dpdy = (f["p"][:, 2:, :] - f["p"][:, :-2, :]) / 2.0
    assert np.max(np.abs(dpdy[:, 2:-2, :] - expected)) < 1e-12 * 9e-5
    assert np.max(np.abs(np.stack([f["ux"], f["uy"], f["uz"]]))) < 1e-15
