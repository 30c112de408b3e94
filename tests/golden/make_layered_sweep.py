"""Writes layered_sweep_8x256_oracle.txt: steady layered Poiseuille profiles of the
FP64 oracle for the 8 x 256 channel (walls in y, fluid A in the lower half),
density ratios {1, 10, 100, 1000} x dynamic viscosity ratios {1, 10, 100},
F_x = 1e-7, step viscosity model for density ratio != 1 (Sec. 4.3, Eq. 37
setting), each case run until u_x changes by less than 2e-6 of its maximum
over 50 000 steps (at most 4 000 000 steps).

Only the oracle computes here; the workload module supplies the parameters and
the initial tanh profile (Eq. 9). Run from the repository root:
    python tests/golden/make_layered_sweep.py [processes]
(about an hour on 8 cores: one single-threaded oracle per case).
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "layered_sweep_8x256_oracle.txt")
CHUNK, MAX_STEPS, STOP = 50000, 4000000, 2e-6


def eq37(cfg, ny):
    h = ny / 2.0
    muA, muB = cfg["rho_A"] * cfg["nu_A"], cfg["rho_B"] * cfg["nu_B"]
    G = cfg["force_x"]
    y = np.arange(ny) + 0.5 - ny / 2
    mu_up, mu_dn = muB, muA               # A below: the upper layer is fluid B
    r = y / h
    a = (mu_up - mu_dn) / (mu_up + mu_dn)
    return np.where(y > 0, G * h * h / (2 * mu_up) * (-r * r - r * a + 2 * mu_up / (mu_up + mu_dn)),
                    G * h * h / (2 * mu_dn) * (-r * r - r * a + 2 * mu_dn / (mu_up + mu_dn)))


def run_case(args):
    rr, mr = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_1902_08933_gb300 import workloads as wl
    cfg = wl.layered_poiseuille(rho_ratio=rr, mu_ratio=mr, viscosity=0 if rr == 1.0 else 1)
    P = orc.params(cfg)
    st = orc.init(P, wl.initial_phi(cfg))
    prev, steps = None, 0
    while steps < MAX_STEPS:
        orc.step(P, st, CHUNK)
        steps += CHUNK
        ux = orc.fields(P, st)["ux"][:, 0].copy()
        if prev is not None and np.max(np.abs(ux - prev)) < STOP * np.max(np.abs(ux)):
            break
        prev = ux
    ua = eq37(cfg, cfg["ny"])
    err = float(np.abs(ux - ua).sum() / np.abs(ua).sum())
    return rr, mr, steps, err, ux


def main():
    nproc = int(sys.argv[1]) if len(sys.argv) > 1 else os.cpu_count()
    cases = [(rr, mr) for rr in (1.0, 10.0, 100.0, 1000.0) for mr in (1.0, 10.0, 100.0)]
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(run_case, cases)
    with open(OUT, "w") as f:
        f.write("# Steady u_x(y) of the FP64 oracle, 8 x 256 layered Poiseuille channel\n"
                "# (Sec. 4.3 setting, Eq. 37 analytic profile; x periodic, halfway bounce-back\n"
                "# walls in y, A below, W = 4, sigma = 0.001, tau_h = 1, F_x = 1e-7, the less\n"
                "# viscous fluid at tau = 0.6, M_phi = min(0.1, 0.2 / gamma), QIM).\n"
                "# Written by tests/golden/make_layered_sweep.py (oracle only).\n"
                "# Each case: one line 'case rho_ratio mu_ratio steps l1_error_vs_eq37',\n"
                "# then 256 values of u_x, y = 0 .. 255.\n")
        for rr, mr, steps, err, ux in res:
            f.write("case %g %g %d %.6e\n" % (rr, mr, steps, err))
            for k in range(0, len(ux), 8):
                f.write(" ".join("%.9e" % v for v in ux[k:k + 8]) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
