"""Pins of the oracles of Remarks 3, 1, 2 and 4 (Sec. 2.3). Remark 3: the generalized model with
rho~ = rho_0 and constant density, the incompressible Navier-Stokes equations
with a mass source (div u = S).

Checked against the moment conditions the remark's equilibrium and force term
must meet (App. A with rho = 1), pressure recovery from Eq. 28, a closed-form
steady flow with a sinusoidal mass source (div u = S fixes u; second-order
convergence), the body-force Poiseuille profile with S = 0 (Guo's model, as
the remark notes), and exact translation equivariance.
"""
import numpy as np
import pytest

CS2 = 1.0 / 3.0
RNG = np.random.default_rng(33)
C = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=float)


def test_remark3_equilibrium_moments(orc):
    for rho0 in (0.0, 1.0):
        for _ in range(4):
            p = RNG.uniform(-1e-2, 1e-2)
            u = RNG.uniform(-0.05, 0.05, 2)
            g = orc.sp_geq(p, u[0], u[1], rho0)
            assert np.isclose(g.sum(), rho0, atol=1e-15)
            assert np.allclose(g @ C, u, atol=1e-16)
            assert np.allclose(np.einsum("i,ia,ib->ab", g, C, C), p * np.eye(2) + np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("xi", [0.0, 0.05])
def test_remark3_force_moments(orc, xi):
    P = orc.sp_params(dict(nx=4, ny=4, nu=0.1, xi=xi))
    tau = 0.1 / CS2 + 0.5
    Q = CS2 - xi / (tau - 0.5)
    for _ in range(4):
        S = RNG.uniform(-1e-3, 1e-3)
        F = RNG.uniform(-1e-4, 1e-4, 2)
        u = RNG.uniform(-0.05, 0.05, 2)
        G = orc.sp_force(P, S, F[0], F[1], u[0], u[1])
        assert np.isclose(G.sum(), S, atol=1e-18)
        assert np.allclose(G @ C, F, atol=1e-18)
        M2 = np.einsum("i,ia,ib->ab", G, C, C)
        assert np.allclose(M2, CS2 * S * np.eye(2) + np.outer(u, F) + np.outer(F, u) + Q * S * np.eye(2),
                           atol=1e-18)


def test_remark3_pressure_recovery(orc):
    # g = g^eq(p, u), F = 0: Eq. 28 returns p + c_s^2/(1 - w_0) (S/2 + (tau - 1/2) G_0)
    P = orc.sp_params(dict(nx=4, ny=4, nu=0.1))
    tau = 0.1 / CS2 + 0.5
    for _ in range(4):
        p, S = RNG.uniform(-1e-2, 1e-2), RNG.uniform(-1e-3, 1e-3)
        u = RNG.uniform(-0.05, 0.05, 2)
        g = orc.sp_geq(p, u[0], u[1], 0.0)
        ux, uy, pout = orc.sp_moments(P, g, S)
        G0 = orc.sp_force(P, S, 0.0, 0.0, u[0], u[1])[0]
        assert np.allclose([ux, uy], u, atol=1e-17)
        assert np.isclose(pout, p + 0.6 * (0.5 * S + (tau - 0.5) * G0), atol=1e-16)


def _source_flow_error(orc, nx, steps=80000):
    P = orc.sp_params(dict(nx=nx, ny=2, nu=0.1))
    k, A = 2 * np.pi / nx, 1e-4
    x = np.arange(nx)
    S = np.tile(A * np.sin(k * x), (2, 1))
    g = orc.sp_init(P)
    orc.sp_step(P, S, g, steps)
    f = orc.sp_fields(P, S, g)
    ua = -(A / k) * np.cos(k * x)              # div u = S, zero mean momentum
    return np.max(np.abs(f["ux"][0] - ua)) / np.max(np.abs(ua)), f


def test_mass_source_flow_closed_form(orc):
    e32, f32 = _source_flow_error(orc, 32)
    e64, _ = _source_flow_error(orc, 64)
    assert np.abs(f32["uy"]).max() == 0.0
    assert e64 < 1e-3
    assert 3.5 < e32 / e64 < 4.5               # second order in space


def test_poiseuille_without_source(orc):
    # S = 0: Guo's incompressible model; body-force Poiseuille flow between
    # halfway walls at y = -1/2 and ny - 1/2. BGK with halfway bounce-back
    # reproduces the parabola exactly at tau = 1/2 + sqrt(3/16) (elsewhere the
    # walls slip by a tau-dependent multiple of F)
    ny, F = 24, 1e-6
    nu = CS2 * np.sqrt(3.0 / 16.0)
    P = orc.sp_params(dict(nx=2, ny=ny, walls_y=1, nu=nu, force_x=F))
    S = np.zeros((ny, 2))
    g = orc.sp_init(P)
    orc.sp_step(P, S, g, 30000)
    ux = orc.sp_fields(P, S, g)["ux"][:, 0]
    y = np.arange(ny)
    ua = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-11


def test_translation_equivariance_sp(orc):
    P = orc.sp_params(dict(nx=12, ny=10, nu=0.05, force_x=1e-5, force_y=-2e-5))
    S = RNG.uniform(-1e-3, 1e-3, (10, 12))
    a, b = orc.sp_init(P), orc.sp_init(P)
    orc.sp_step(P, S, a, 20)
    orc.sp_step(P, np.roll(S, (3, 5), axis=(0, 1)), b, 20)
    assert np.array_equal(np.roll(a, (3, 5), axis=(1, 2)), b)


# ---------------------------------------------------------------- Remark 1
def test_remark1_equilibrium_and_force_moments(orc):
    P = orc.sp_params(dict(nx=4, ny=4, nu=0.1, xi=0.02, force_x=3e-5, force_y=-1e-5))
    tau = 0.1 / CS2 + 0.5
    F = np.array([3e-5, -1e-5])
    for _ in range(4):
        rho = RNG.uniform(0.8, 1.2)
        u = RNG.uniform(-0.05, 0.05, 2)
        geq = orc.sp1_geq(rho, u[0], u[1])
        assert np.isclose(geq.sum(), rho, atol=1e-15)                                   # Eq. 29bb moments
        assert np.allclose(geq @ C, rho * u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", geq, C, C), rho * CS2 * np.eye(2) + rho * np.outer(u, u),
                           atol=1e-15)
        S, divu = RNG.uniform(-1e-3, 1e-3), RNG.uniform(-1e-3, 1e-3)
        G = orc.sp1_force(P, S, rho, u[0], u[1], divu)
        Q = rho * CS2 - 0.02 / (tau - 0.5)
        assert np.isclose(G.sum(), S, atol=1e-18)
        assert np.allclose(G @ C, F, atol=1e-18)
        M2 = np.einsum("i,ia,ib->ab", G, C, C)
        expect = (CS2 * S * np.eye(2) + np.outer(u, F) + np.outer(F, u) - np.outer(u, u) * S
                  + Q * divu * np.eye(2))
        assert np.allclose(M2, expect, atol=1e-18)


def test_remark1_mass_balance(orc):
    # rho = sum g + S/2 (Eq. 27aa) and sum G = S: the total mass grows by sum S a step
    P = orc.sp_params(dict(nx=16, ny=12, nu=0.08, walls_y=1, force_x=1e-6))
    S = np.ascontiguousarray(RNG.uniform(0, 2e-5, (12, 16)))
    g = orc.sp1_init(P, 1.0)
    m0 = orc.sp1_fields(P, S, g)["rho"].sum()
    orc.sp1_step(P, S, g, 50)
    m1 = orc.sp1_fields(P, S, g)["rho"].sum()
    assert abs(m1 - m0 - 50 * S.sum()) < 1e-12 * m0


def test_remark1_mass_source_flow(orc):
    errs = []
    for nx in (32, 64):
        P = orc.sp_params(dict(nx=nx, ny=2, nu=0.1))
        k, A = 2 * np.pi / nx, 1e-4
        x = np.arange(nx)
        S = np.tile(A * np.sin(k * x), (2, 1))
        g = orc.sp1_init(P, 1.0)
        orc.sp1_step(P, S, g, 80000)
        f = orc.sp1_fields(P, S, g)
        ua = -(A / k) * np.cos(k * x)
        errs.append(np.max(np.abs(f["ux"][0] - ua)) / np.max(np.abs(ua)))
    assert errs[1] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5


# ---------------------------------------------------------------- Remark 4
def _drag(F0, lam, beta, u):
    return F0 - (lam + beta * np.linalg.norm(u)) * u


def test_remark4_uniform_state_is_adams_bashforth(orc):
    # a uniform state under F(u) = F0 - (lambda + beta|u|) u: sum c f_eq = u and
    # sum c G = F, so the Remark 4 update of the momentum is u + F(u_n) +
    # [F(u_n) - F(u_{n-1})]/2, the two-step Adams-Bashforth rule for du/dt = F(u)
    # (first step Euler: G at t = -1 is G at t = 0)
    lam, beta, F0 = 0.01, 0.5, np.array([1e-4, -5e-5])
    P = orc.sp_params(dict(nx=4, ny=3, nu=0.1, force_x=F0[0], force_y=F0[1], drag_lin=lam, drag_quad=beta))
    S = np.zeros((3, 4))
    f, G = orc.sp4_init(P, S)
    u, up = np.zeros(2), np.zeros(2)
    for _ in range(60):
        orc.sp4_step(P, S, f, G, 1)
        u, up = u + 1.5 * _drag(F0, lam, beta, u) - 0.5 * _drag(F0, lam, beta, up), u
        r = orc.sp4_fields(P, S, f)
        assert np.allclose(r["ux"], u[0], rtol=0, atol=1e-17) and np.allclose(r["uy"], u[1], rtol=0, atol=1e-17)


def test_remark4_uniform_drag_steady_state(orc):
    # steady: F(u) = 0, |u| = (-lambda + sqrt(lambda^2 + 4 beta |F0|)) / (2 beta) along F0
    lam, beta, F0 = 0.02, 2.0, np.array([3e-5, 4e-5])
    P = orc.sp_params(dict(nx=3, ny=2, nu=0.1, force_x=F0[0], force_y=F0[1], drag_lin=lam, drag_quad=beta))
    S = np.zeros((2, 3))
    f, G = orc.sp4_init(P, S)
    orc.sp4_step(P, S, f, G, 5000)
    r = orc.sp4_fields(P, S, f)
    mag = (-lam + np.sqrt(lam * lam + 4 * beta * np.linalg.norm(F0))) / (2 * beta)
    ue = mag * F0 / np.linalg.norm(F0)
    assert np.allclose(r["ux"], ue[0], rtol=1e-12) and np.allclose(r["uy"], ue[1], rtol=1e-12)


def test_remark4_hydrostatic_rest(orc):
    # walls in y, a uniform force towards a wall: the fluid stays at rest and
    # grad p = F exactly (bounce-back acts on g = f - G/2)
    ny, Fy = 16, -1e-5
    P = orc.sp_params(dict(nx=2, ny=ny, walls_y=1, nu=0.1, force_y=Fy))
    S = np.zeros((ny, 2))
    f, G = orc.sp4_init(P, S)
    orc.sp4_step(P, S, f, G, 20000)
    r = orc.sp4_fields(P, S, f)
    assert np.abs(r["uy"]).max() < 1e-15 and np.abs(r["ux"]).max() < 1e-15
    assert np.allclose(np.diff(r["p"][:, 0]), Fy, rtol=1e-9, atol=0)


def test_remark4_poiseuille_exact_at_the_magic_tau(orc):
    ny, F = 24, 1e-6
    nu = CS2 * np.sqrt(3.0 / 16.0)
    P = orc.sp_params(dict(nx=2, ny=ny, walls_y=1, nu=nu, force_x=F))
    S = np.zeros((ny, 2))
    f, G = orc.sp4_init(P, S)
    orc.sp4_step(P, S, f, G, 30000)
    ux = orc.sp4_fields(P, S, f)["ux"][:, 0]
    y = np.arange(ny)
    ua = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-11


def test_remark4_brinkman_second_order(orc):
    # -nu u'' + lambda u = F between walls at y = +-H: u = (F/lambda)(1 - cosh(ky)/cosh(kH)),
    # k = sqrt(lambda/nu); lambda scaled with 1/ny^2 keeps kH fixed while refining
    def err(ny, steps):
        nu, F, lam = 0.1, 1e-5, 1.6 / ny ** 2
        P = orc.sp_params(dict(nx=2, ny=ny, walls_y=1, nu=nu, force_x=F, drag_lin=lam))
        S = np.zeros((ny, 2))
        f, G = orc.sp4_init(P, S)
        orc.sp4_step(P, S, f, G, steps)
        ux = orc.sp4_fields(P, S, f)["ux"][:, 0]
        y = np.arange(ny) + 0.5 - ny / 2
        k = np.sqrt(lam / nu)
        ua = F / lam * (1 - np.cosh(k * y) / np.cosh(k * ny / 2))
        return np.abs(ux - ua).max() / ua.max()
    e16, e32 = err(16, 40000), err(32, 80000)
    assert e32 < 2e-3 and 3.0 < e16 / e32 < 5.0


def test_remark4_source_flow_with_drag(orc):
    # div u = S fixes u = -(A/k) cos kx; the linear drag removes the mean momentum
    errs = []
    for nx in (32, 64):
        P = orc.sp_params(dict(nx=nx, ny=2, nu=0.1, drag_lin=0.002))
        k, A = 2 * np.pi / nx, 1e-4
        x = np.arange(nx)
        S = np.tile(A * np.sin(k * x), (2, 1))
        f, G = orc.sp4_init(P, S)
        orc.sp4_step(P, S, f, G, 80000)
        r = orc.sp4_fields(P, S, f)
        assert np.abs(r["uy"]).max() == 0.0
        ua = -(A / k) * np.cos(k * x)
        errs.append(np.max(np.abs(r["ux"][0] - ua)) / np.max(np.abs(ua)))
    assert errs[1] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5


def test_remark4_translation_equivariance(orc):
    P = orc.sp_params(dict(nx=12, ny=10, nu=0.05, force_x=1e-5, force_y=-2e-5, drag_lin=0.01, drag_quad=0.3))
    S = RNG.uniform(-1e-3, 1e-3, (10, 12))
    a, Ga = orc.sp4_init(P, S)
    Sb = np.roll(S, (3, 5), axis=(0, 1))
    b, Gb = orc.sp4_init(P, Sb)
    orc.sp4_step(P, S, a, Ga, 20)
    orc.sp4_step(P, Sb, b, Gb, 20)
    assert np.array_equal(np.roll(a, (3, 5), axis=(1, 2)), b)


# ---------------------------------------------------------------- Remark 2
def test_remark2_equilibrium_and_force_moments(orc):
    p0, xi, nu = 0.4, 0.02, 0.1
    F1 = np.array([3e-5, -1e-5])
    P = orc.sp_params(dict(nx=4, ny=4, nu=nu, xi=xi, force_x=F1[0], force_y=F1[1], p0=p0))
    tau = nu / CS2 + 0.5
    for _ in range(4):
        p = p0 + RNG.uniform(-1e-3, 1e-3)
        u = RNG.uniform(-0.05, 0.05, 2)
        geq = orc.sp2_geq(p, p0, u[0], u[1])                                           # Eq. 29bd
        assert np.isclose(geq.sum(), p, atol=1e-15)
        assert np.allclose(geq @ C, p0 * u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", geq, C, C), p * CS2 * np.eye(2) + p0 * np.outer(u, u),
                           atol=1e-15)
        S1, divu = RNG.uniform(-1e-3, 1e-3), RNG.uniform(-1e-3, 1e-3)
        G = orc.sp2_force(P, S1, u[0], u[1], divu)
        Q2 = p0 * CS2 - xi / (tau - 0.5)
        assert np.isclose(G.sum(), p0 * S1, atol=1e-18)
        assert np.allclose(G @ C, p0 * F1, atol=1e-18)
        expect = CS2 * p0 * S1 * np.eye(2) + p0 * (np.outer(u, F1) + np.outer(F1, u)) + Q2 * divu * np.eye(2)
        assert np.allclose(np.einsum("i,ia,ib->ab", G, C, C), expect, atol=1e-18)


def test_remark2_pressure_balance(orc):
    # p = sum g + p0 S1 / 2 and sum G = p0 S1: the sum of p grows by p0 sum S1 a step
    P = orc.sp_params(dict(nx=16, ny=12, nu=0.08, walls_y=1, force_x=1e-6, p0=0.5))
    S1 = np.ascontiguousarray(RNG.uniform(0, 2e-5, (12, 16)))
    g = orc.sp2_init(P)
    m0 = orc.sp2_fields(P, S1, g)["p"].sum()
    orc.sp2_step(P, S1, g, 50)
    m1 = orc.sp2_fields(P, S1, g)["p"].sum()
    assert abs(m1 - m0 - 50 * 0.5 * S1.sum()) < 1e-12 * m0


def test_remark2_source_flow_and_p0_invariance(orc):
    # div u = S1 fixes u = -(A/k) cos kx, second order; u does not depend on p0 (xi = 0)
    errs = []
    for nx in (32, 64):
        k, A = 2 * np.pi / nx, 1e-4
        x = np.arange(nx)
        S1 = np.tile(A * np.sin(k * x), (2, 1))
        P = orc.sp_params(dict(nx=nx, ny=2, nu=0.1, p0=1.0 / 3.0))
        g = orc.sp2_init(P)
        orc.sp2_step(P, S1, g, 80000)
        f = orc.sp2_fields(P, S1, g)
        ua = -(A / k) * np.cos(k * x)
        errs.append(np.max(np.abs(f["ux"][0] - ua)) / np.max(np.abs(ua)))
        if nx == 32:
            P2 = orc.sp_params(dict(nx=nx, ny=2, nu=0.1, p0=2.0))
            g2 = orc.sp2_init(P2)
            orc.sp2_step(P2, S1, g2, 2000)
            g1 = orc.sp2_init(P)
            orc.sp2_step(P, S1, g1, 2000)
            a, b = orc.sp2_fields(P2, S1, g2)["ux"], orc.sp2_fields(P, S1, g1)["ux"]
            assert np.abs(a - b).max() < 1e-10 * np.abs(b).max()   # rounding only
    assert errs[1] < 1e-3 and 3.5 < errs[0] / errs[1] < 4.5


def test_remark2_poiseuille_exact_at_the_magic_tau(orc):
    # S1 = 0: the incompressible model of He et al.; halfway bounce-back exact at tau = 1/2 + sqrt(3/16)
    ny, F = 24, 1e-6
    nu = CS2 * np.sqrt(3.0 / 16.0)
    P = orc.sp_params(dict(nx=2, ny=ny, walls_y=1, nu=nu, force_x=F, p0=1.0))
    S1 = np.zeros((ny, 2))
    g = orc.sp2_init(P)
    orc.sp2_step(P, S1, g, 30000)
    ux = orc.sp2_fields(P, S1, g)["ux"][:, 0]
    y = np.arange(ny)
    ua = F / (2 * nu) * (y + 0.5) * (ny - 0.5 - y)
    assert np.max(np.abs(ux - ua)) / ua.max() < 1e-11
