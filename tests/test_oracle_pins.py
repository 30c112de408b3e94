"""Pins of the FP64 oracle's building blocks against closed forms.

Each check is an identity the paper or the lattice fixes (moment conditions of
App. A, Eq. a23 and Eqs. a25aa / a25aaa; lattice isotropy of Sec. 2.2; the
inverse of Eqs. 6-7; Fourier symbols of the stencils of Eq. 30), so a dropped
term, a wrong sign, a wrong weight or a transposed operand in the oracle fails
at least one of them.
"""
import itertools

import numpy as np
import pytest

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(20190822)


def lat(orc):
    cx, cy, w, op = orc.lattice()
    c = np.stack([cx, cy], axis=1).astype(float)
    return c, w, op


def test_lattice_isotropy(orc):
    c, w, op = lat(orc)
    assert np.isclose(w.sum(), 1.0, rtol=0, atol=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-15)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, CS2 * np.eye(2), atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(third, 0.0, atol=1e-15)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(2)
    expect = CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                         + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(fourth, expect, atol=1e-15)
    # opposite directions
    for i in range(9):
        assert np.array_equal(c[op[i]], -c[i])
    # rest direction first, then the four axis and the four diagonal directions
    assert np.array_equal(c[0], [0, 0])
    assert all(np.abs(c[i]).sum() == 1 for i in range(1, 5))
    assert all(np.abs(c[i]).sum() == 2 for i in range(5, 9))


def test_derived_parameters_invert_eqs_6_7(orc):
    for sigma, W in [(0.001, 4.0), (0.03, 4.0), (0.0922, 5.0), (1.7, 3.0)]:
        P = orc.params(dict(nx=4, ny=4, rho_A=10, rho_B=1, nu_A=.1, nu_B=.1, sigma=sigma, W=W,
                            tau_h=0.8, M=0.02))
        D = orc.derive(P)
        assert np.isclose(np.sqrt(8 * D.kappa / D.beta), W, rtol=1e-14)      # Eq. 6
        assert np.isclose(np.sqrt(2 * D.kappa * D.beta) / 6, sigma, rtol=1e-14)  # Eq. 7
        assert np.isclose(D.eta * CS2 * (0.8 - 0.5), 0.02, rtol=1e-14)       # Eq. 17
        assert np.isclose(D.gamma, 9.0, rtol=1e-15)   # (rho_A - rho_B) / rho_B with phi_A=1, phi_B=0
    P = orc.params(dict(nx=4, ny=4, rho_A=2, rho_B=2, nu_A=.1, nu_B=.1, sigma=.01, W=4, tau_h=1, M=.1))
    assert orc.derive(P).gamma == 0.0


def test_equilibrium_planar_profile_has_zero_chemical_potential():
    # Eq. 9 minimises the free energy of Eqs. 4-5 when beta, kappa follow Eqs. 6-7:
    # 4 beta phi (phi-1)(phi-1/2) - kappa phi'' = 0 for phi = 1/2 + 1/2 tanh(2z/W).
    sigma, W = 0.01, 4.0
    kappa, beta = 1.5 * sigma * W, 12 * sigma / W
    z = np.linspace(-10, 10, 201)
    t = np.tanh(2 * z / W)
    phi = 0.5 + 0.5 * t
    d2 = 0.5 * (2 / W) ** 2 * (-2 * t * (1 - t ** 2))
    mu = 4 * beta * phi * (phi - 1) * (phi - 0.5) - kappa * d2
    assert np.max(np.abs(mu)) < 1e-15


def test_s_moments(orc):
    c, w, _ = lat(orc)
    for _ in range(20):
        u = RNG.normal(scale=0.05, size=2)
        s = np.array([orc.s(i, *u) for i in range(9)])
        assert abs(s.sum()) < 1e-16
        assert np.allclose(s @ c, u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", s, c, c), np.outer(u, u), atol=1e-16)


@pytest.mark.parametrize("rho0", [0.0, 1.0, 7.5])
def test_geq_moments_eq33(orc, rho0):
    # App. A, Eq. a23 and below: M0 = rho~, M1 = rho u, M2 = p I + rho u u.
    c, w, _ = lat(orc)
    for _ in range(20):
        p = RNG.normal(scale=1e-3)
        rho = RNG.uniform(0.5, 100)
        u = RNG.normal(scale=0.05, size=2)
        geq = orc.geq(p, rho, *u, rho0)
        assert np.isclose(geq.sum(), rho0, rtol=0, atol=1e-13 * max(1, rho))
        assert np.allclose(geq @ c, rho * u, rtol=0, atol=1e-13 * rho)
        m2 = np.einsum("i,ia,ib->ab", geq, c, c)
        assert np.allclose(m2, p * np.eye(2) + rho * np.outer(u, u), rtol=0, atol=1e-13 * rho)


def test_heq_moments_eq11(orc):
    c, w, _ = lat(orc)
    for _ in range(20):
        phi = RNG.uniform(-0.1, 1.1)
        mu = RNG.normal(scale=1e-3)
        eta = RNG.uniform(0.1, 2)
        u = RNG.normal(scale=0.05, size=2)
        heq = orc.heq(phi, mu, eta, *u)
        assert np.isclose(heq.sum(), phi, rtol=0, atol=1e-15)                       # Eq. 18
        assert np.allclose(heq @ c, phi * u, rtol=0, atol=1e-16)
        m2 = np.einsum("i,ia,ib->ab", heq, c, c)
        assert np.allclose(m2, eta * mu * CS2 * np.eye(2), rtol=0, atol=1e-16)    # gives M = eta c_s^2 (tau-1/2)


def test_force_distribution_moments_eq34(orc):
    # sum G = S (Eq. a23), sum c G = F (Eq. a25aa), and
    # sum c c G = c_s^2 S I + u F~ + F~ u + (2/d) rho c_s^2 S1 I (Eq. a25aaa with the
    # d_t p and u u S~ terms dropped and xi = 0, Sec. 3.2.1).
    c, w, _ = lat(orc)
    for _ in range(30):
        rho = RNG.uniform(0.5, 100)
        S1 = RNG.normal(scale=1e-4)
        u = RNG.normal(scale=0.05, size=2)
        F = RNG.normal(scale=1e-4, size=2)
        Ft = RNG.normal(scale=1e-4, size=2)
        S = RNG.normal(scale=1e-4)
        G = orc.force_dist(S, rho, S1, *F, *Ft, *u)
        assert np.isclose(G.sum(), S, rtol=0, atol=1e-18 + 1e-13 * abs(S))
        assert np.allclose(G @ c, F, rtol=0, atol=1e-17)
        m2 = np.einsum("i,ia,ib->ab", G, c, c)
        expect = CS2 * S * np.eye(2) + np.outer(u, Ft) + np.outer(Ft, u) + rho * CS2 * S1 * np.eye(2)
        assert np.allclose(m2, expect, rtol=0, atol=1e-17 + 1e-13 * np.abs(expect).max())


def test_printed_G0_vs_eq34_at_rest_direction(orc):
    # Reading Q1: Eq. 34 at i = 0 gives omega_0 [u.grad(rho) - u.F~ / c_s^2]
    # = -omega_0 u.(F - grad p) / c_s^2; the printed simplification adds
    # omega_0 (1 - 1/d) rho S1.
    w0 = 4.0 / 9.0
    for _ in range(30):
        rho = RNG.uniform(0.5, 100)
        S1 = RNG.normal(scale=1e-4)
        u = RNG.normal(scale=0.05, size=2)
        F = RNG.normal(scale=1e-4, size=2)
        gradp = RNG.normal(scale=1e-4, size=2)
        gradrho = RNG.normal(scale=1e-2, size=2)
        S = u @ gradrho + rho * S1
        Ft = F - gradp + CS2 * gradrho
        G0_lit = orc.force_dist(S, rho, S1, *F, *Ft, *u)[0]
        G0_pr = orc.G0_printed(rho, S1, *F, *gradp, *u)
        assert np.isclose(G0_lit, -w0 * (u @ (F - gradp)) / CS2, rtol=1e-9, atol=1e-20)
        assert np.isclose(G0_pr - G0_lit, w0 * 0.5 * rho * S1, rtol=1e-7, atol=1e-19)
        if S1 == 0.0:
            assert G0_pr == G0_lit


def test_source_R_moments_eq14(orc):
    c, w, _ = lat(orc)
    for tau in (0.6, 0.8, 1.0, 1.7):
        d = RNG.normal(scale=1e-5, size=2)
        R = orc.source_R(tau, *d)
        assert abs(R.sum()) < 1e-20
        assert np.allclose(R @ c, (1 - 1 / (2 * tau)) * d, rtol=1e-13, atol=0)


def test_pressure_recovers_p_from_equilibrium(orc):
    # With g = g^eq(p, u) (Eq. 33): sum_{i!=0} g_i = (1 - w0) p / c_s^2 - rho s_0(u), so
    # Eq. 29 returns p + c_s^2 S / (2 (1 - w0)) = p + 0.3 S, and Eq. 28 adds
    # c_s^2 / (1 - w0) (tau_g - 1/2) G_0 = 0.6 (tau_g - 1/2) G_0.
    for _ in range(30):
        p = RNG.normal(scale=1e-3)
        rho = RNG.uniform(0.5, 100)
        u = RNG.normal(scale=0.05, size=2)
        S = RNG.normal(scale=1e-4)
        G0 = RNG.normal(scale=1e-5)
        tau = RNG.uniform(0.51, 3)
        g = orc.geq(p, rho, *u, RNG.uniform(0, 2))
        assert np.isclose(orc.pressure(2, g, 0.0, rho, *u, tau, G0), p, rtol=0, atol=1e-13 * rho)
        assert np.isclose(orc.pressure(2, g, S, rho, *u, tau, G0), p + 0.3 * S, rtol=0, atol=1e-13 * rho)
        for scheme in (0, 1):
            assert np.isclose(orc.pressure(scheme, g, S, rho, *u, tau, G0),
                              p + 0.3 * S + 0.6 * (tau - 0.5) * G0, rtol=0, atol=1e-13 * rho)


def test_tau_g_viscosity_models(orc):
    base = dict(nx=4, ny=4, rho_A=10.0, rho_B=1.0, nu_A=0.2, nu_B=0.05, sigma=.01, W=4,
                tau_h=1, M=.1)
    P = orc.params(base, viscosity=0)
    assert np.isclose(orc.tau_g(P, 1.0, 10.0), 3 * 0.2 + 0.5, rtol=1e-15)
    assert np.isclose(orc.tau_g(P, 0.0, 1.0), 3 * 0.05 + 0.5, rtol=1e-15)
    harmonic = 1.0 / (0.5 / 0.2 + 0.5 / 0.05)
    assert np.isclose(orc.tau_g(P, 0.5, 5.5), 3 * harmonic + 0.5, rtol=1e-14)
    P = orc.params(base, viscosity=1)
    assert np.isclose(orc.tau_g(P, 0.5, 5.0), 3 * (10.0 * 0.2 / 5.0) + 0.5, rtol=1e-15)
    assert np.isclose(orc.tau_g(P, 0.49, 5.0), 3 * (1.0 * 0.05 / 5.0) + 0.5, rtol=1e-15)


def _grid(nx, ny, walls=0):
    from oracle import oracle as o
    return o.params(dict(nx=nx, ny=ny, walls_y=walls, rho_A=1, rho_B=1, nu_A=.1, nu_B=.1,
                         sigma=.01, W=4, tau_h=1, M=.1))


def test_stencil_fourier_symbols_eq30(orc):
    # On a periodic grid f = sin(k.x): Eq. 30b gives [6 sum w_i (cos(k.c_i) - 1)] f and
    # Eq. 30a gives cos(k.x) * 3 sum w_i c_i sin(k.c_i); both tend to -|k|^2 f and k cos(k.x).
    c, w, _ = lat(orc)
    nx, ny = 24, 18
    P = _grid(nx, ny)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    for mx, my in [(1, 0), (0, 1), (2, 3), (5, 4), (11, 8)]:
        k = np.array([2 * np.pi * mx / nx, 2 * np.pi * my / ny])
        f = np.sin(k[0] * X + k[1] * Y)
        lam = 6 * np.sum(w * (np.cos(c @ k) - 1))
        assert np.allclose(orc.lap(P, f), lam * f, atol=1e-13)
        gx, gy = orc.grad(P, f)
        sym = 3 * (w * np.sin(c @ k)) @ c
        cosf = np.cos(k[0] * X + k[1] * Y)
        assert np.allclose(gx, sym[0] * cosf, atol=1e-13)
        assert np.allclose(gy, sym[1] * cosf, atol=1e-13)
    # second-order consistency for a long wave
    k = np.array([2 * np.pi / nx, 0.0])
    lam = 6 * np.sum(w * (np.cos(c @ k) - 1))
    assert abs(lam / -(k @ k) - 1) < 0.01


def test_stencil_exact_on_polynomials_interior(orc):
    nx, ny = 16, 16
    P = _grid(nx, ny)
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    f = 0.3 * X - 0.7 * Y + 2.0
    gx, gy = orc.grad(P, f)
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(gx[inner], 0.3, atol=1e-13) and np.allclose(gy[inner], -0.7, atol=1e-13)
    f = X ** 2 + 2 * X * Y - 3 * Y ** 2
    assert np.allclose(orc.lap(P, f)[inner], 2 - 6, atol=1e-12)


def test_wall_stencil_is_mirror_extension(orc):
    # Reading Q7: next to a wall the stencils see the field mirrored about the wall.
    # Equivalent: the periodic stencil on the grid doubled by reflection in y.
    nx, ny = 7, 9
    f = RNG.normal(size=(ny, nx))
    Pw = _grid(nx, ny, walls=1)
    ext = np.concatenate([f, f[::-1]], axis=0)
    Pp = _grid(nx, 2 * ny, walls=0)
    assert np.allclose(orc.lap(Pw, f), orc.lap(Pp, ext)[:ny], atol=1e-14)
    gxw, gyw = orc.grad(Pw, f)
    gxp, gyp = orc.grad(Pp, ext)
    assert np.allclose(gxw, gxp[:ny], atol=1e-14) and np.allclose(gyw, gyp[:ny], atol=1e-14)


def test_streaming_periodic_and_bounce_back(orc):
    c, w, op = lat(orc)
    nx, ny = 5, 6
    for walls in (0, 1):
        P = _grid(nx, ny, walls)
        for i, (x, y) in itertools.product(range(9), [(0, 0), (2, 3), (4, 5), (1, 5)]):
            post = np.zeros((9, ny, nx))
            post[i, y, x] = 1.0
            pre = orc.stream(P, post)
            assert pre.sum() == 1.0
            tx, ty = x + int(c[i, 0]), y + int(c[i, 1])
            if walls and not (0 <= ty < ny):
                assert pre[op[i], y, x] == 1.0      # halfway bounce-back: back at x, reversed
            else:
                assert pre[i, ty % ny, tx % nx] == 1.0


def test_layered_profile_eq37_closed_form(orc):
    # Eq. 37: continuous velocity and shear stress at the interface, no slip at both walls,
    # and the single-fluid parabola when mu_up = mu_down.
    h, G = 50.0, 3e-7
    for mu_up, mu_down in [(0.1, 0.3), (1.0, 10.0), (0.5, 0.5)]:
        u = lambda y: orc.layered_ux(y, h, G, mu_up, mu_down)
        assert abs(u(h)) < 1e-18 and abs(u(-h)) < 1e-18
        e = 1e-6
        assert np.isclose(u(e), u(-e), rtol=1e-6)
        s_up = mu_up * (u(2 * e) - u(e)) / e
        s_dn = mu_down * (u(-e) - u(-2 * e)) / e
        assert np.isclose(s_up, s_dn, rtol=1e-4)
        # momentum balance: mu u'' = -G on each side
        y = 0.3 * h
        assert np.isclose(mu_up * (u(y + 1e-3) - 2 * u(y) + u(y - 1e-3)) / 1e-6, -G, rtol=1e-4)
    assert np.isclose(orc.layered_ux(10.0, h, G, 0.5, 0.5), G / (2 * 0.5) * (h * h - 100.0), rtol=1e-14)
