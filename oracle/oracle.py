"""ctypes binding of the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module. It shares nothing with the CUDA
path; the only thing both sides take in common is the seeded input recipe of
``paper_1902_08933_gb300.workloads`` (parameter dictionaries and initial order
parameter fields), which holds none of the method's arithmetic.

Arrays: float64, C-contiguous, grid arrays shaped (ny, nx), population arrays
shaped (9, ny, nx) in the D2Q9 order of Sec. 2.2 of arXiv:1902.08933.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
SRC3 = os.path.join(HERE, "oracle3d.c")
SRCSP = os.path.join(HERE, "oracle_sp.c")
HDR = os.path.join(HERE, "oracle.h")
# Two builds of the same sources: the parity build (default; FP contraction off,
# so a*b+c rounds twice exactly as written) and, with LBM_ORACLE_BUILD=timed,
# an -O3 build that only the CPU timing legs of the benchmark load (its results
# may differ from the parity build's by rounding; it is never compared with).
TIMED = os.environ.get("LBM_ORACLE_BUILD", "parity") == "timed"
LIB = os.path.join(HERE, "liboracle_timed.so" if TIMED else "liboracle.so")
_FLAGS = (["-O3", "-std=gnu11"] if TIMED else
          ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11"])

_lock = threading.Lock()
_lib = None

_DP = ctypes.POINTER(ctypes.c_double)


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` in oracle.h (field order matters)."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("walls_y", ctypes.c_int),
        ("qim", ctypes.c_int), ("pressure", ctypes.c_int), ("surface_force", ctypes.c_int),
        ("viscosity", ctypes.c_int),
        ("rho_A", ctypes.c_double), ("rho_B", ctypes.c_double),
        ("nu_A", ctypes.c_double), ("nu_B", ctypes.c_double),
        ("sigma", ctypes.c_double), ("W", ctypes.c_double),
        ("tau_h", ctypes.c_double), ("M", ctypes.c_double),
        ("force_x", ctypes.c_double), ("force_y", ctypes.c_double),
        ("gravity", ctypes.c_double), ("rho0", ctypes.c_double),
    ]


class Derived(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kappa", ctypes.c_double),
                ("eta", ctypes.c_double), ("gamma", ctypes.c_double)]


class Diag(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "sum_phi", "sum_rho", "kinetic_energy", "max_u",
        "centroid_A_x", "centroid_A_y", "centroid_B_x", "centroid_B_y",
        "mass_A", "mass_B", "P_bulk_A", "P_bulk_B", "n_bulk_A", "n_bulk_B")] + [
        ("nonfinite", ctypes.c_int)]


class SpParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("walls_y", ctypes.c_int),
                ("nu", ctypes.c_double), ("xi", ctypes.c_double), ("force_x", ctypes.c_double),
                ("force_y", ctypes.c_double), ("rho0", ctypes.c_double), ("drag_lin", ctypes.c_double),
                ("drag_quad", ctypes.c_double), ("p0", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle library with gcc (the parity build unless
    LBM_ORACLE_BUILD=timed). Rebuilds when the sources are newer than it."""
    with _lock:
        stale = (not os.path.exists(LIB) or
                 os.path.getmtime(LIB) < max(os.path.getmtime(SRC), os.path.getmtime(SRC3),
                                             os.path.getmtime(SRCSP), os.path.getmtime(HDR)))
        if force or stale:
            tmp = LIB + ".tmp.%d" % os.getpid()
            cmd = (["gcc"] + _FLAGS + ["-fopenmp", "-fPIC", "-shared", SRC, SRC3, SRCSP,
                                       "-o", tmp, "-lm"])
            subprocess.run(cmd, check=True)
            os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        P = ctypes.POINTER(Params)
        L.orc_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  _DP, ctypes.POINTER(ctypes.c_int)]
        L.orc_derive.argtypes = [P, ctypes.POINTER(Derived)]
        L.orc_s.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.orc_s.restype = ctypes.c_double
        L.orc_geq.argtypes = [ctypes.c_double] * 5 + [_DP]
        L.orc_heq.argtypes = [ctypes.c_double] * 5 + [_DP]
        L.orc_force_dist.argtypes = [ctypes.c_double] * 9 + [_DP]
        L.orc_G0_printed.argtypes = [ctypes.c_double] * 8
        L.orc_G0_printed.restype = ctypes.c_double
        L.orc_source_R.argtypes = [ctypes.c_double] * 3 + [_DP]
        L.orc_pressure.argtypes = [ctypes.c_int, _DP] + [ctypes.c_double] * 6
        L.orc_pressure.restype = ctypes.c_double
        L.orc_tau_g.argtypes = [P, ctypes.c_double, ctypes.c_double]
        L.orc_tau_g.restype = ctypes.c_double
        L.orc_grad.argtypes = [P, _DP, _DP, _DP]
        L.orc_lap.argtypes = [P, _DP, _DP]
        L.orc_stream.argtypes = [P, _DP, _DP]
        L.orc_init.argtypes = [P, _DP, _DP, _DP, _DP, _DP]
        L.orc_step.argtypes = [P, _DP, _DP, _DP, _DP, ctypes.c_int]
        L.orc_fields.argtypes = [P, _DP, _DP, _DP] + [_DP] * 7
        L.orc_diagnostics.argtypes = [P, _DP, _DP, _DP, ctypes.POINTER(Diag)]
        L.orc_layered_ux.argtypes = [ctypes.c_double] * 5
        L.orc_layered_ux.restype = ctypes.c_double
        IP = ctypes.POINTER(ctypes.c_int)
        L.orc3_lattice.argtypes = [IP, IP, IP, _DP, IP]
        L.orc3_s.argtypes = [ctypes.c_int, _DP]
        L.orc3_s.restype = ctypes.c_double
        L.orc3_geq.argtypes = [ctypes.c_double, ctypes.c_double, _DP, ctypes.c_double, _DP]
        L.orc3_heq.argtypes = [ctypes.c_double] * 3 + [_DP, _DP]
        L.orc3_force_dist.argtypes = [ctypes.c_double] * 3 + [_DP] * 4
        L.orc3_G0_printed.argtypes = [ctypes.c_double, ctypes.c_double, _DP, _DP, _DP]
        L.orc3_G0_printed.restype = ctypes.c_double
        L.orc3_source_R.argtypes = [ctypes.c_double, _DP, _DP]
        L.orc3_pressure.argtypes = [ctypes.c_int, _DP, ctypes.c_double, ctypes.c_double, _DP,
                                    ctypes.c_double, ctypes.c_double]
        L.orc3_pressure.restype = ctypes.c_double
        L.orc3_grad.argtypes = [P, ctypes.c_int, _DP, _DP, _DP, _DP]
        L.orc3_lap.argtypes = [P, ctypes.c_int, _DP, _DP]
        L.orc3_stream.argtypes = [P, ctypes.c_int, _DP, _DP]
        L.orc3_init.argtypes = [P, ctypes.c_int, _DP, _DP, _DP, _DP, _DP]
        L.orc3_step.argtypes = [P, ctypes.c_int, _DP, _DP, _DP, _DP, ctypes.c_int]
        L.orc3_fields.argtypes = [P, ctypes.c_int, _DP, _DP, _DP] + [_DP] * 8
        L.orc3_diagnostics.argtypes = [P, ctypes.c_int, _DP, _DP, _DP, ctypes.POINTER(Diag)]
        SP = ctypes.POINTER(SpParams)
        L.orc_sp_tau.argtypes = [SP]
        L.orc_sp_tau.restype = ctypes.c_double
        L.orc_sp_geq.argtypes = [ctypes.c_double] * 4 + [_DP]
        L.orc_sp_force.argtypes = [SP] + [ctypes.c_double] * 5 + [_DP]
        L.orc_sp_moments.argtypes = [SP, _DP, ctypes.c_double, _DP, _DP, _DP]
        L.orc_sp_init.argtypes = [SP, _DP]
        L.orc_sp_step.argtypes = [SP, _DP, _DP, ctypes.c_int]
        L.orc_sp_fields.argtypes = [SP, _DP, _DP, _DP, _DP, _DP]
        L.orc_sp1_moments.argtypes = [SP, _DP, ctypes.c_double, _DP, _DP, _DP]
        L.orc_sp1_force.argtypes = [SP] + [ctypes.c_double] * 5 + [_DP]
        L.orc_sp1_geq.argtypes = [ctypes.c_double] * 3 + [_DP]
        L.orc_sp1_init.argtypes = [SP, ctypes.c_double, _DP]
        L.orc_sp1_step.argtypes = [SP, _DP, _DP, ctypes.c_int]
        L.orc_sp2_moments.argtypes = [SP, _DP, ctypes.c_double, _DP, _DP, _DP]
        L.orc_sp2_force.argtypes = [SP] + [ctypes.c_double] * 4 + [_DP]
        L.orc_sp2_geq.argtypes = [ctypes.c_double] * 4 + [_DP]
        L.orc_sp2_init.argtypes = [SP, _DP]
        L.orc_sp2_step.argtypes = [SP, _DP, _DP, ctypes.c_int]
        L.orc_sp2_fields.argtypes = [SP, _DP, _DP, _DP, _DP, _DP]
        L.orc_sp4_moments.argtypes = [SP, _DP, ctypes.c_double, _DP, _DP, _DP]
        L.orc_sp4_init.argtypes = [SP, _DP, _DP, _DP]
        L.orc_sp4_step.argtypes = [SP, _DP, _DP, _DP, ctypes.c_int]
        L.orc_sp4_fields.argtypes = [SP, _DP, _DP, _DP, _DP, _DP]
        L.orc_sp1_fields.argtypes = [SP, _DP, _DP, _DP, _DP, _DP]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


_INT_KEYS = ("nx", "ny", "walls_y", "qim", "pressure", "surface_force", "viscosity")
_DBL_KEYS = ("rho_A", "rho_B", "nu_A", "nu_B", "sigma", "W", "tau_h", "M",
             "force_x", "force_y", "gravity", "rho0")


def params(cfg: dict, **over) -> Params:
    """Build ``orc_params`` from a workload dictionary (missing keys default to 0)."""
    d = dict(cfg)
    d.update(over)
    P = Params()
    for k in _INT_KEYS:
        setattr(P, k, int(d.get(k, 0)))
    for k in _DBL_KEYS:
        setattr(P, k, float(d.get(k, 0.0)))
    return P


# ---------------------------------------------------------------- building blocks
def lattice():
    L = lib()
    cx = (ctypes.c_int * 9)()
    cy = (ctypes.c_int * 9)()
    w = (ctypes.c_double * 9)()
    op = (ctypes.c_int * 9)()
    L.orc_lattice(cx, cy, w, op)
    return np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(op[:])


def derive(P: Params) -> Derived:
    D = Derived()
    if lib().orc_derive(ctypes.byref(P), ctypes.byref(D)):
        raise ValueError("invalid parameters")
    return D


def s(i, ux, uy):
    return lib().orc_s(i, ux, uy)


def geq(p, rho, ux, uy, rho0=0.0):
    out = np.zeros(9)
    lib().orc_geq(p, rho, ux, uy, rho0, _ptr(out))
    return out


def heq(phi, mu, eta, ux, uy):
    out = np.zeros(9)
    lib().orc_heq(phi, mu, eta, ux, uy, _ptr(out))
    return out


def force_dist(S, rho, S1, Fx, Fy, Ftx, Fty, ux, uy):
    out = np.zeros(9)
    lib().orc_force_dist(S, rho, S1, Fx, Fy, Ftx, Fty, ux, uy, _ptr(out))
    return out


def G0_printed(rho, S1, Fx, Fy, dpx, dpy, ux, uy):
    return lib().orc_G0_printed(rho, S1, Fx, Fy, dpx, dpy, ux, uy)


def source_R(tau_h, dx, dy):
    out = np.zeros(9)
    lib().orc_source_R(tau_h, dx, dy, _ptr(out))
    return out


def pressure(scheme, g, S, rho, ux, uy, tau_g, G0):
    g = np.ascontiguousarray(g, dtype=np.float64)
    return lib().orc_pressure(scheme, _ptr(g), S, rho, ux, uy, tau_g, G0)


def tau_g(P: Params, phi, rho):
    return lib().orc_tau_g(ctypes.byref(P), phi, rho)


def grad(P: Params, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    gx = np.zeros_like(f)
    gy = np.zeros_like(f)
    lib().orc_grad(ctypes.byref(P), _ptr(f), _ptr(gx), _ptr(gy))
    return gx, gy


def lap(P: Params, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    lib().orc_lap(ctypes.byref(P), _ptr(f), _ptr(out))
    return out


def stream(P: Params, post):
    post = np.ascontiguousarray(post, dtype=np.float64)
    pre = np.zeros_like(post)
    lib().orc_stream(ctypes.byref(P), _ptr(post), _ptr(pre))
    return pre


def layered_ux(y, hh, G, mu_up, mu_down):
    return lib().orc_layered_ux(y, hh, G, mu_up, mu_down)


# ---------------------------------------------------------------- whole grid
def init(P: Params, phi0) -> dict:
    ny, nx = P.ny, P.nx
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(ny, nx)
    st = {"h": np.zeros((9, ny, nx)), "g": np.zeros((9, ny, nx)),
          "phiu_prev": np.zeros((2, ny, nx)), "p_prev": np.zeros((ny, nx))}
    rc = lib().orc_init(ctypes.byref(P), _ptr(phi0), _ptr(st["h"]), _ptr(st["g"]),
                        _ptr(st["phiu_prev"]), _ptr(st["p_prev"]))
    if rc:
        raise ValueError("orc_init failed (%d)" % rc)
    return st


def step(P: Params, st: dict, n: int) -> dict:
    rc = lib().orc_step(ctypes.byref(P), _ptr(st["h"]), _ptr(st["g"]),
                        _ptr(st["phiu_prev"]), _ptr(st["p_prev"]), int(n))
    if rc:
        raise ValueError("orc_step failed (%d)" % rc)
    return st


def fields(P: Params, st: dict) -> dict:
    ny, nx = P.ny, P.nx
    out = {k: np.zeros((ny, nx)) for k in ("phi", "ux", "uy", "p", "rho", "mu", "P")}
    rc = lib().orc_fields(ctypes.byref(P), _ptr(st["h"]), _ptr(st["g"]), _ptr(st["p_prev"]),
                          *[_ptr(out[k]) for k in ("phi", "ux", "uy", "p", "rho", "mu", "P")])
    if rc:
        raise ValueError("orc_fields failed (%d)" % rc)
    return out


def diagnostics(P: Params, st: dict) -> dict:
    D = Diag()
    rc = lib().orc_diagnostics(ctypes.byref(P), _ptr(st["h"]), _ptr(st["g"]),
                               _ptr(st["p_prev"]), ctypes.byref(D))
    if rc:
        raise ValueError("orc_diagnostics failed (%d)" % rc)
    return {k: getattr(D, k) for k, _ in Diag._fields_}


def run(cfg: dict, phi0, nsteps: int, **over):
    """Initialise from phi0 and advance nsteps; returns (params, state)."""
    P = params(cfg, **over)
    st = init(P, phi0)
    if nsteps:
        step(P, st, nsteps)
    return P, st


# ---------------------------------------------------------------- D3Q15 (3-D)
def lattice3():
    """D3Q15 velocities, weights and opposite directions (Sec. 2.2)."""
    cx, cy, cz, op = (ctypes.c_int * 15)(), (ctypes.c_int * 15)(), (ctypes.c_int * 15)(), (ctypes.c_int * 15)()
    w = np.zeros(15)
    lib().orc3_lattice(cx, cy, cz, _ptr(w), op)
    return np.array([list(cx), list(cy), list(cz)]), w, np.array(list(op))


def _v3(u):
    a = np.ascontiguousarray(u, dtype=np.float64)
    assert a.shape == (3,)
    return a


def s3(i, u):
    return lib().orc3_s(i, _ptr(_v3(u)))


def geq3(p, rho, u, rho0=0.0):
    out = np.zeros(15)
    lib().orc3_geq(p, rho, _ptr(_v3(u)), rho0, _ptr(out))
    return out


def heq3(phi, mu, eta, u):
    out = np.zeros(15)
    lib().orc3_heq(phi, mu, eta, _ptr(_v3(u)), _ptr(out))
    return out


def force_dist3(S, rho, S1, F, Ft, u):
    out = np.zeros(15)
    lib().orc3_force_dist(S, rho, S1, _ptr(_v3(F)), _ptr(_v3(Ft)), _ptr(_v3(u)), _ptr(out))
    return out


def G0_printed3(rho, S1, F, dp, u):
    return lib().orc3_G0_printed(rho, S1, _ptr(_v3(F)), _ptr(_v3(dp)), _ptr(_v3(u)))


def source_R3(tau_h, dphiu):
    out = np.zeros(15)
    lib().orc3_source_R(tau_h, _ptr(_v3(dphiu)), _ptr(out))
    return out


def pressure3(scheme, g, S, rho, u, tau_g, G0):
    return lib().orc3_pressure(scheme, _ptr(np.ascontiguousarray(g, dtype=np.float64)), S, rho,
                               _ptr(_v3(u)), tau_g, G0)


def grad3(P: Params, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    gx, gy, gz = np.zeros_like(f), np.zeros_like(f), np.zeros_like(f)
    lib().orc3_grad(ctypes.byref(P), f.shape[0], _ptr(f), _ptr(gx), _ptr(gy), _ptr(gz))
    return gx, gy, gz


def lap3(P: Params, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    lib().orc3_lap(ctypes.byref(P), f.shape[0], _ptr(f), _ptr(out))
    return out


def stream3(P: Params, post):
    post = np.ascontiguousarray(post, dtype=np.float64)
    out = np.zeros_like(post)
    lib().orc3_stream(ctypes.byref(P), post.shape[1], _ptr(post), _ptr(out))
    return out


def init3(P: Params, phi0) -> dict:
    """State of a D3Q15 grid from phi0 of shape (nz, ny, nx)."""
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    nz, ny, nx = phi0.shape
    assert (ny, nx) == (P.ny, P.nx)
    st = {"nz": nz, "h": np.zeros((15, nz, ny, nx)), "g": np.zeros((15, nz, ny, nx)),
          "phiu_prev": np.zeros((3, nz, ny, nx)), "p_prev": np.zeros((nz, ny, nx))}
    rc = lib().orc3_init(ctypes.byref(P), nz, _ptr(phi0), _ptr(st["h"]), _ptr(st["g"]),
                         _ptr(st["phiu_prev"]), _ptr(st["p_prev"]))
    if rc:
        raise ValueError("orc3_init failed (%d)" % rc)
    return st


def step3(P: Params, st: dict, n: int) -> dict:
    rc = lib().orc3_step(ctypes.byref(P), st["nz"], _ptr(st["h"]), _ptr(st["g"]),
                         _ptr(st["phiu_prev"]), _ptr(st["p_prev"]), int(n))
    if rc:
        raise ValueError("orc3_step failed (%d)" % rc)
    return st


def fields3(P: Params, st: dict) -> dict:
    shape = st["p_prev"].shape
    names = ("phi", "ux", "uy", "uz", "p", "rho", "mu", "P")
    out = {k: np.zeros(shape) for k in names}
    rc = lib().orc3_fields(ctypes.byref(P), st["nz"], _ptr(st["h"]), _ptr(st["g"]), _ptr(st["p_prev"]),
                           *[_ptr(out[k]) for k in names])
    if rc:
        raise ValueError("orc3_fields failed (%d)" % rc)
    return out


def diagnostics3(P: Params, st: dict) -> dict:
    D = Diag()
    rc = lib().orc3_diagnostics(ctypes.byref(P), st["nz"], _ptr(st["h"]), _ptr(st["g"]),
                                _ptr(st["p_prev"]), ctypes.byref(D))
    if rc:
        raise ValueError("orc3_diagnostics failed (%d)" % rc)
    return {k: getattr(D, k) for k, _ in Diag._fields_}


# ------------------------------------------------- single-phase model of Remark 3
def sp_params(cfg: dict) -> SpParams:
    P = SpParams()
    P.nx, P.ny, P.walls_y = int(cfg["nx"]), int(cfg["ny"]), int(cfg.get("walls_y", 0))
    P.nu, P.xi = float(cfg["nu"]), float(cfg.get("xi", 0.0))
    P.force_x, P.force_y = float(cfg.get("force_x", 0.0)), float(cfg.get("force_y", 0.0))
    P.rho0 = float(cfg.get("rho0", 0.0))
    P.drag_lin, P.drag_quad = float(cfg.get("drag_lin", 0.0)), float(cfg.get("drag_quad", 0.0))
    P.p0 = float(cfg.get("p0", 1.0 / 3.0))
    return P


def sp_geq(p, ux, uy, rho0=0.0):
    out = np.zeros(9)
    lib().orc_sp_geq(p, ux, uy, rho0, _ptr(out))
    return out


def sp_force(P: SpParams, S, Fx, Fy, ux, uy):
    out = np.zeros(9)
    lib().orc_sp_force(ctypes.byref(P), S, Fx, Fy, ux, uy, _ptr(out))
    return out


def sp_moments(P: SpParams, g, S):
    ux, uy, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_sp_moments(ctypes.byref(P), _ptr(np.ascontiguousarray(g, dtype=np.float64)), S,
                         ctypes.cast(ctypes.byref(ux), _DP), ctypes.cast(ctypes.byref(uy), _DP),
                         ctypes.cast(ctypes.byref(p), _DP))
    return ux.value, uy.value, p.value


def sp_init(P: SpParams) -> np.ndarray:
    g = np.zeros((9, P.ny, P.nx))
    lib().orc_sp_init(ctypes.byref(P), _ptr(g))
    return g


def sp_step(P: SpParams, S, g, n: int):
    S = np.ascontiguousarray(S, dtype=np.float64)
    rc = lib().orc_sp_step(ctypes.byref(P), _ptr(S), _ptr(g), int(n))
    if rc:
        raise ValueError("orc_sp_step failed (%d)" % rc)
    return g


def sp_fields(P: SpParams, S, g) -> dict:
    S = np.ascontiguousarray(S, dtype=np.float64)
    out = {k: np.zeros((P.ny, P.nx)) for k in ("ux", "uy", "p")}
    lib().orc_sp_fields(ctypes.byref(P), _ptr(S), _ptr(g), _ptr(out["ux"]), _ptr(out["uy"]), _ptr(out["p"]))
    return out


# ------------------------------------------------- Remark 1 (nearly incompressible)
def sp1_geq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_sp1_geq(rho, ux, uy, _ptr(out))
    return out


def sp1_force(P: SpParams, S, rho, ux, uy, divu):
    out = np.zeros(9)
    lib().orc_sp1_force(ctypes.byref(P), S, rho, ux, uy, divu, _ptr(out))
    return out


def sp1_init(P: SpParams, rho_init=1.0) -> np.ndarray:
    g = np.zeros((9, P.ny, P.nx))
    lib().orc_sp1_init(ctypes.byref(P), rho_init, _ptr(g))
    return g


def sp1_step(P: SpParams, S, g, n: int):
    S = np.ascontiguousarray(S, dtype=np.float64)
    rc = lib().orc_sp1_step(ctypes.byref(P), _ptr(S), _ptr(g), int(n))
    if rc:
        raise ValueError("orc_sp1_step failed (%d)" % rc)
    return g


def sp1_fields(P: SpParams, S, g) -> dict:
    S = np.ascontiguousarray(S, dtype=np.float64)
    out = {k: np.zeros((P.ny, P.nx)) for k in ("rho", "ux", "uy")}
    lib().orc_sp1_fields(ctypes.byref(P), _ptr(S), _ptr(g), _ptr(out["rho"]), _ptr(out["ux"]), _ptr(out["uy"]))
    return out


# ------------------------------------------------- Remark 4 (explicit D_i G_i)
def sp4_moments(P: SpParams, f, S):
    ux, uy, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().orc_sp4_moments(ctypes.byref(P), _ptr(np.ascontiguousarray(f, dtype=np.float64)), S,
                          ctypes.cast(ctypes.byref(ux), _DP), ctypes.cast(ctypes.byref(uy), _DP),
                          ctypes.cast(ctypes.byref(p), _DP))
    return ux.value, uy.value, p.value


def sp4_init(P: SpParams, S):
    """(f, Gprev): f at rest, Gprev = G of that state (standing in for t = -1)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    f, G = np.zeros((9, P.ny, P.nx)), np.zeros((9, P.ny, P.nx))
    lib().orc_sp4_init(ctypes.byref(P), _ptr(S), _ptr(f), _ptr(G))
    return f, G


def sp4_step(P: SpParams, S, f, Gprev, n: int):
    S = np.ascontiguousarray(S, dtype=np.float64)
    rc = lib().orc_sp4_step(ctypes.byref(P), _ptr(S), _ptr(f), _ptr(Gprev), int(n))
    if rc:
        raise ValueError("orc_sp4_step failed (%d)" % rc)
    return f


def sp4_fields(P: SpParams, S, f) -> dict:
    S = np.ascontiguousarray(S, dtype=np.float64)
    out = {k: np.zeros((P.ny, P.nx)) for k in ("ux", "uy", "p")}
    lib().orc_sp4_fields(ctypes.byref(P), _ptr(S), _ptr(f), _ptr(out["ux"]), _ptr(out["uy"]), _ptr(out["p"]))
    return out


# ------------------------------------------------- Remark 2 (He-type, source S_1)
def sp2_geq(p, p0, ux, uy):
    out = np.zeros(9)
    lib().orc_sp2_geq(p, p0, ux, uy, _ptr(out))
    return out


def sp2_force(P: SpParams, S1, ux, uy, divu):
    out = np.zeros(9)
    lib().orc_sp2_force(ctypes.byref(P), S1, ux, uy, divu, _ptr(out))
    return out


def sp2_init(P: SpParams) -> np.ndarray:
    g = np.zeros((9, P.ny, P.nx))
    lib().orc_sp2_init(ctypes.byref(P), _ptr(g))
    return g


def sp2_step(P: SpParams, S1, g, n: int):
    S1 = np.ascontiguousarray(S1, dtype=np.float64)
    rc = lib().orc_sp2_step(ctypes.byref(P), _ptr(S1), _ptr(g), int(n))
    if rc:
        raise ValueError("orc_sp2_step failed (%d)" % rc)
    return g


def sp2_fields(P: SpParams, S1, g) -> dict:
    S1 = np.ascontiguousarray(S1, dtype=np.float64)
    out = {k: np.zeros((P.ny, P.nx)) for k in ("p", "ux", "uy")}
    lib().orc_sp2_fields(ctypes.byref(P), _ptr(S1), _ptr(g), _ptr(out["p"]), _ptr(out["ux"]), _ptr(out["uy"]))
    return out
