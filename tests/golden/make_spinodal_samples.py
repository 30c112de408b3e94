"""Writes spinodal_512_oracle_samples.txt: the FP64 oracle's fields of the 512 x 512
spinodal decomposition (Sec. 4.1 setting; periodic, density ratio 3, sigma =
0.005, W = 4, tau = 0.7, M = 0.1, F_s = mu grad(phi), QIM, phi0 = 1/2 + U[-0.005,
0.005] from splitmix64 seed 1902) after 2000, 5000, 10000 and 20000 steps, at
512 cells drawn with splitmix64 seed 77, plus each field's maximum magnitude over
the whole grid (the normaliser of the field-max error metric).

Only the oracle computes here. Run from the repository root:
    python tests/golden/make_spinodal_samples.py
(several minutes on 8 cores).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "spinodal_512_oracle_samples.txt")
CHECKPOINTS = (2000, 5000, 10000, 20000)
FIELDS = ("phi", "ux", "uy", "p")


def sample_cells(n=512, size=512, seed=77):
    from paper_1902_08933_gb300 import workloads as wl
    u = wl.uniform01(seed, 2 * n).reshape(n, 2)
    return (u[:, 0] * size).astype(int), (u[:, 1] * size).astype(int)   # x, y


def main():
    from oracle import oracle as orc
    from paper_1902_08933_gb300 import workloads as wl
    cfg = wl.spinodal()
    P = orc.params(cfg)
    st = orc.init(P, wl.initial_phi(cfg))
    xs, ys = sample_cells()
    done = 0
    lines = ["# FP64 oracle, 512 x 512 spinodal decomposition (Sec. 4.1 setting, QIM),",
             "# written by tests/golden/make_spinodal_samples.py (oracle only).",
             "# 'step N' blocks: 'max phi ux uy p' (max |field| over the grid), then",
             "# one line per sampled cell: x y phi ux uy p (cells: splitmix64 seed 77)."]
    for n in CHECKPOINTS:
        orc.step(P, st, n - done)
        done = n
        f = orc.fields(P, st)
        lines.append("step %d" % n)
        lines.append("max " + " ".join("%.17e" % np.max(np.abs(f[k])) for k in FIELDS))
        for x, y in zip(xs, ys):
            lines.append("%d %d " % (x, y) + " ".join("%.17e" % f[k][y, x] for k in FIELDS))
        print("step", n, flush=True)
    with open(OUT, "w") as fo:
        fo.write("\n".join(lines) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
