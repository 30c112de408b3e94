"""Seeded synthetic workloads: parameter sets and initial order-parameter fields.

This module is the one piece shared by the CUDA path's callers (tests, bench)
and the CPU oracle. It holds none of the lattice Boltzmann arithmetic: only
the experiment recipes of Sec. 4 of arXiv:1902.08933 (initial droplet / bubble
/ planar / noisy fields and the physical parameters), resized to the benchmark
configurations, and a counter-based random generator for the noise.

A workload is a plain dict of physical parameters (keys of ``PARAM_KEYS``) plus
an ``init`` entry describing phi_0; ``initial_phi(cfg)`` returns phi_0 as a
float64 array of shape (ny, nx).
"""
from __future__ import annotations

import numpy as np

PARAM_KEYS = ("nx", "ny", "walls_y", "qim", "pressure", "surface_force", "viscosity",
              "rho_A", "rho_B", "nu_A", "nu_B", "sigma", "W", "tau_h", "M",
              "force_x", "force_y", "gravity")

# ----------------------------------------------------------------------------------
# splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): a counter-based generator, so the value at a cell
# depends only on (seed, cell index).
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    z = counter.astype(np.uint64) * _GOLDEN + _GOLDEN  # state after (counter+1) increments
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of splitmix64(seed * 2^32 + k)."""
    with np.errstate(over="ignore"):
        k = np.arange(n, dtype=np.uint64) + np.uint64((seed & 0xFFFFFFFF) << 32)
        z = splitmix64(k)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# ----------------------------------------------------------------------------------
# Initial fields (Sec. 4): droplet Eq. 36, planar interface Eq. 9, bubble (the
# droplet profile with the phases swapped, Sec. 4.4), noisy mixture (Sec. 4.1).
def initial_phi(cfg: dict) -> np.ndarray:
    """phi_0 of shape (ny, nx), or (nz, ny, nx) for a D3Q15 workload (nz > 1)."""
    if int(cfg.get("nz", 0)) > 1:
        return _initial_phi3(cfg)
    nx, ny = int(cfg["nx"]), int(cfg["ny"])
    spec = cfg["init"]
    kind = spec["kind"]
    W = float(cfg["W"])
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    if kind in ("droplet", "bubble"):
        r = np.sqrt((x - spec["cx"]) ** 2 + (y - spec["cy"]) ** 2)
        prof = 0.5 + 0.5 * np.tanh(2.0 * (spec["R"] - r) / W)
        phi = prof if kind == "droplet" else 1.0 - prof
    elif kind == "layered":
        # node j sits at y_j = j + 1/2 - ny/2 between walls at -ny/2 and +ny/2;
        # phase A (phi = 1) below the interface when spec["A_below"].
        yc = y + 0.5 - ny / 2.0
        sgn = -1.0 if spec.get("A_below", True) else 1.0
        phi = 0.5 + 0.5 * np.tanh(sgn * 2.0 * yc / W) + 0.0 * x
    elif kind == "noise":
        u = uniform01(int(spec["seed"]), nx * ny).reshape(ny, nx)
        phi = spec["mean"] + spec["amp"] * (2.0 * u - 1.0)
    elif kind == "uniform":
        phi = np.full((ny, nx), float(spec["value"]))
    else:
        raise ValueError("unknown init kind %r" % kind)
    return np.array(np.broadcast_to(phi, (ny, nx)), dtype=np.float64, order="C")


def _initial_phi3(cfg: dict) -> np.ndarray:
    """3-D phi_0: a sphere (Eq. 36 with the 3-D distance), a planar interface
    normal to y (Eq. 9), noise or a uniform field."""
    nx, ny, nz = int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"])
    spec = cfg["init"]
    kind = spec["kind"]
    W = float(cfg["W"])
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    if kind in ("droplet", "bubble"):
        r = np.sqrt((x - spec["cx"]) ** 2 + (y - spec["cy"]) ** 2 + (z - spec["cz"]) ** 2)
        prof = 0.5 + 0.5 * np.tanh(2.0 * (spec["R"] - r) / W)
        phi = prof if kind == "droplet" else 1.0 - prof
    elif kind == "layered":
        yc = y + 0.5 - ny / 2.0
        sgn = -1.0 if spec.get("A_below", True) else 1.0
        phi = 0.5 + 0.5 * np.tanh(sgn * 2.0 * yc / W) + 0.0 * x + 0.0 * z
    elif kind == "noise":
        u = uniform01(int(spec["seed"]), nx * ny * nz).reshape(nz, ny, nx)
        phi = spec["mean"] + spec["amp"] * (2.0 * u - 1.0)
    elif kind == "uniform":
        phi = np.full((nz, ny, nx), float(spec["value"]))
    else:
        raise ValueError("unknown init kind %r" % kind)
    return np.array(np.broadcast_to(phi, (nz, ny, nx)), dtype=np.float64, order="C")


def _nu_from_tau(tau: float) -> float:
    # kinematic viscosity of a BGK fluid with relaxation time tau (c_s^2 = 1/3)
    return (tau - 0.5) / 3.0


# ----------------------------------------------------------------------------------
# The five benchmark configurations (2-D D2Q9). Values not fixed by the
# configuration text follow Sec. 4 of the paper; each such choice is listed in
# the design notes (readings Q3, Q9-Q19).
def static_droplet(n: int = 64, R: float | None = None, rho_ratio: float = 10.0,
                   sigma: float = 0.01, W: float = 4.0, tau_g: float = 0.8,
                   tau_h: float = 0.8, M: float = 0.02, qim: int = 1, pressure: int = 0) -> dict:
    R = n / 4.0 if R is None else R
    nu = _nu_from_tau(tau_g)
    return dict(nx=n, ny=n, walls_y=0, qim=qim, pressure=pressure, surface_force=1,
                viscosity=0, rho_A=rho_ratio, rho_B=1.0, nu_A=nu, nu_B=nu, sigma=sigma,
                W=W, tau_h=tau_h, M=M, force_x=0.0, force_y=0.0, gravity=0.0,
                init=dict(kind="droplet", cx=n / 2.0, cy=n / 2.0, R=R),
                name="static_droplet_%dx%d" % (n, n))


def spinodal(n: int = 512, seed: int = 1902, qim: int = 1, pressure: int = 0) -> dict:
    nu = _nu_from_tau(0.7)
    return dict(nx=n, ny=n, walls_y=0, qim=qim, pressure=pressure, surface_force=0,
                viscosity=0, rho_A=3.0, rho_B=1.0, nu_A=nu, nu_B=nu, sigma=0.005, W=4.0,
                tau_h=0.7, M=0.1, force_x=0.0, force_y=0.0, gravity=0.0,
                init=dict(kind="noise", seed=seed, mean=0.5, amp=0.005),
                name="spinodal_%dx%d" % (n, n))


def layered_poiseuille(nx: int = 8, ny: int = 256, rho_ratio: float = 1.0,
                       mu_ratio: float = 1.0, force_x: float = 1e-7, viscosity: int = 0,
                       tau_min: float = 0.6, qim: int = 1, sigma: float = 0.001,
                       M: float = 0.1, tau_h: float = 1.0) -> dict:
    """Phase A (phi = 1) in the lower half, B above, walls in y. mu_ratio is the
    dynamic ratio mu_A / mu_B; the less viscous fluid (kinematic) gets tau_min.
    M is capped by stable_mobility (unchanged for rho_ratio <= 3)."""
    rho_A, rho_B = rho_ratio, 1.0
    M = stable_mobility(M, rho_A, rho_B)
    # mu_A = mu_ratio * mu_B; nu = mu / rho
    nuA_over_nuB = mu_ratio * rho_B / rho_A
    nu_min = _nu_from_tau(tau_min)
    if nuA_over_nuB >= 1.0:
        nu_B, nu_A = nu_min, nu_min * nuA_over_nuB
    else:
        nu_A, nu_B = nu_min, nu_min / nuA_over_nuB
    return dict(nx=nx, ny=ny, walls_y=1, qim=qim, pressure=0, surface_force=0,
                viscosity=viscosity, rho_A=rho_A, rho_B=rho_B, nu_A=nu_A, nu_B=nu_B,
                sigma=sigma, W=4.0, tau_h=tau_h, M=M, force_x=force_x, force_y=0.0,
                gravity=0.0, init=dict(kind="layered", A_below=True),
                name="layered_%dx%d_r%g_m%g" % (nx, ny, rho_ratio, mu_ratio))


def stable_mobility(M: float, rho_A: float, rho_B: float) -> float:
    """Mobility capped at 0.2 / gamma, gamma = (rho_A - rho_B) / rho_B: the explicit
    QIM mass source S1 = -gamma M lap(mu) made light-bubble runs diverge (already
    in the FP64 oracle) for gamma M >~ 0.5 (reading Q10)."""
    gamma = abs(rho_A - rho_B) / rho_B
    return M if gamma == 0 else min(M, 0.2 / gamma)


def rising_bubble(nx: int = 1024, ny: int = 4096, R: float = 128.0, cy: float = 512.0,
                  rho_ratio: float = 10.0, Eo: float = 10.0, Re: float = 35.0,
                  U_g: float = 0.01, W: float = 5.0, qim: int = 1, M: float = 0.1,
                  tau_h: float = 1.0) -> dict:
    """Light bubble (phase B) in heavy ambient A, walls at top and bottom,
    periodic sides. D = 2R, U_g = sqrt(g D): g = U_g^2 / D,
    sigma = g (rho_A - rho_B) D^2 / Eo, nu = U_g D / Re in both phases (reading Q19);
    M capped by stable_mobility."""
    D = 2.0 * R
    g = U_g * U_g / D
    rho_A, rho_B = rho_ratio, 1.0
    sigma = g * (rho_A - rho_B) * D * D / Eo
    nu = U_g * D / Re
    M = stable_mobility(M, rho_A, rho_B)
    return dict(nx=nx, ny=ny, walls_y=1, qim=qim, pressure=0, surface_force=0,
                viscosity=0, rho_A=rho_A, rho_B=rho_B, nu_A=nu, nu_B=nu, sigma=sigma,
                W=W, tau_h=tau_h, M=M, force_x=0.0, force_y=0.0, gravity=g,
                init=dict(kind="bubble", cx=nx / 2.0, cy=cy, R=R),
                name="bubble_%dx%d_r%g" % (nx, ny, rho_ratio))


def batched_mixed(n_instances: int = 512, seed: int = 4242) -> list:
    """Independent static droplets and rising bubbles on square grids drawn from
    {32, 64, 128, 256}, R = N/4, W = 4, density ratio from {2, 10, 100},
    sigma uniform in [0.001, 0.02], tau_g = tau_h = 0.8; droplets periodic with
    M = 0.02, bubbles walled in y with M = 0.1 and gravity from Eo = 10; M capped
    by stable_mobility."""
    u = uniform01(seed, 4 * n_instances).reshape(n_instances, 4)
    sizes = (32, 64, 128, 256)
    ratios = (2.0, 10.0, 100.0)
    out = []
    nu = _nu_from_tau(0.8)
    for k in range(n_instances):
        N = sizes[min(3, int(u[k, 0] * 4))]
        bubble = u[k, 1] >= 0.5
        ratio = ratios[min(2, int(u[k, 2] * 3))]
        sigma = 0.001 + 0.019 * u[k, 3]
        R = N / 4.0
        M_cap = stable_mobility(1.0, ratio, 1.0)
        cfg = dict(nx=N, ny=N, qim=1, pressure=0, viscosity=0, rho_A=ratio, rho_B=1.0,
                   nu_A=nu, nu_B=nu, sigma=sigma, W=4.0, tau_h=0.8, force_x=0.0, force_y=0.0)
        if bubble:
            D = 2.0 * R
            cfg.update(walls_y=1, surface_force=0, M=min(0.1, M_cap),
                       gravity=10.0 * sigma / ((ratio - 1.0) * D * D),
                       init=dict(kind="bubble", cx=N / 2.0, cy=0.3 * N, R=R),
                       name="batch%03d_bubble_%d_r%g" % (k, N, ratio))
        else:
            cfg.update(walls_y=0, surface_force=1, M=min(0.02, M_cap), gravity=0.0,
                       init=dict(kind="droplet", cx=N / 2.0, cy=N / 2.0, R=R),
                       name="batch%03d_droplet_%d_r%g" % (k, N, ratio))
        out.append(cfg)
    return out


def lups(cfgs, steps: int) -> float:
    """Lattice updates (one cell advanced one step, both population sets)."""
    if isinstance(cfgs, dict):
        cfgs = [cfgs]
    return float(sum(int(c["nx"]) * int(c["ny"]) for c in cfgs)) * steps


def laplace_dp_expected(cfg: dict) -> float:
    """Laplace's law of Sec. 4.2, dP = sigma / R (2-D)."""
    return float(cfg["sigma"]) / float(cfg["init"]["R"])


# ----------------------------------------------------------------------------------
# Three-dimensional (D3Q15) workloads: the same physics with nz planes, x and z
# periodic, walls (if any) normal to y.
def static_droplet3(n: int = 32, R: float | None = None, rho_ratio: float = 10.0,
                    sigma: float = 0.01, W: float = 4.0, tau_g: float = 0.8, tau_h: float = 0.8,
                    M: float = 0.02, qim: int = 1, pressure: int = 0) -> dict:
    """Sphere of phase A in phase B, periodic cube (Sec. 4.2 set-up in 3-D;
    Laplace's law reads Delta p = 2 sigma / R)."""
    cfg = static_droplet(n=n, R=R, rho_ratio=rho_ratio, sigma=sigma, W=W, tau_g=tau_g,
                         tau_h=tau_h, M=M, qim=qim, pressure=pressure)
    cfg["nz"] = n
    cfg["init"] = dict(kind="droplet", cx=n / 2.0, cy=n / 2.0, cz=n / 2.0, R=cfg["init"]["R"])
    cfg["name"] = "droplet3_%d_r%g" % (n, rho_ratio)
    return cfg


def layered_poiseuille3(nx: int = 4, ny: int = 64, nz: int = 4, **kw) -> dict:
    """The layered channel of Sec. 4.3 with nz periodic planes in z."""
    cfg = layered_poiseuille(nx=nx, ny=ny, **kw)
    cfg["nz"] = nz
    cfg["name"] = "layered3_%dx%dx%d" % (nx, ny, nz)
    return cfg


def rising_bubble3(nx: int = 128, ny: int = 256, nz: int = 128, R: float = 24.0,
                   cy: float = 64.0, **kw) -> dict:
    """Light sphere in heavy fluid between walls normal to y (the rising-bubble
    set-up of Sec. 4.4 in 3-D; parameters from Eo and Re as in 2-D)."""
    cfg = rising_bubble(nx=nx, ny=ny, R=R, cy=cy, **kw)
    cfg["nz"] = nz
    cfg["init"] = dict(kind="bubble", cx=nx / 2.0, cy=cy, cz=nz / 2.0, R=R)
    cfg["name"] = "bubble3_%dx%dx%d_r%g" % (nx, ny, nz, cfg["rho_A"])
    return cfg


def laplace_dp_expected3(cfg: dict) -> float:
    """Laplace's law for a sphere, Delta p = 2 sigma / R."""
    return 2.0 * float(cfg["sigma"]) / float(cfg["init"]["R"])
