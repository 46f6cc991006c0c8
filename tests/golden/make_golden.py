"""Writes the stored oracle values used by the GPU tests whose oracle cost is
too high to recompute in a test run (k = 7, all 1024 states summed: about
8e10 FLOP per point).  Calls only the oracle and the seeded input generator.

    python tests/golden/make_golden.py            # |M|^2 and kappa, 512 points
    python tests/golden/make_golden.py --grad     # dual-number gradient, 4 points

The gradient file takes the first points of the |M|^2 file: the oracle's
|M|^2 and d|M|^2/d k_j (3-momenta of the 7 outgoing photons, energies on
shell), one forward-mode dual-number evaluation per component (21 per point).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2511_19456_b300 import phasespace as ps  # noqa: E402

K7_FILE = os.path.join(HERE, "k7_summed_oracle.txt")
K7_GRAD_FILE = os.path.join(HERE, "k7_summed_grad_oracle.txt")
K7_GRAD_POINTS = 4


def main():
    w = ps.WORKLOADS["compton_k7"]
    n = 512
    mom = ps.points(w["k"], n, w["omega"], w["seed"] + 17)
    m2, kap = oracle.m2(mom, kappa=True)
    with open(K7_FILE, "w") as f:
        f.write("# e- gamma -> e- + 7 gamma, omega = 10 m_e, RAMBO points (seeded), all 1024\n")
        f.write("# helicity/polarisation states summed; |M|^2 and kappa from the brute-force FP64\n")
        f.write("# oracle (oracle/qed_oracle.cpp), written by tests/golden/make_golden.py.\n")
        f.write("# per point: one line m2 kappa, then 10 lines E px py pz (slots 0..9)\n")
        for i in range(n):
            f.write(f"{m2[i]:.17e} {kap[i]:.17e}\n")
            for s in range(w["k"] + 3):
                f.write(" ".join(f"{x:.17e}" for x in mom[i, s]) + "\n")


def load_k7():
    rows = [l.split() for l in open(K7_FILE) if l.strip() and not l.startswith("#")]
    k = 7
    per = k + 4
    n = len(rows) // per
    m2 = np.array([float(rows[i * per][0]) for i in range(n)])
    kap = np.array([float(rows[i * per][1]) for i in range(n)])
    mom = np.array([[[float(x) for x in rows[i * per + 1 + s]] for s in range(k + 3)] for i in range(n)])
    return mom, m2, kap


def main_grad(n=K7_GRAD_POINTS):
    mom, _, _ = load_k7()
    mom = np.ascontiguousarray(mom[:n])
    m2, g = oracle.grad(mom)
    k = 7
    with open(K7_GRAD_FILE, "w") as f:
        f.write("# e- gamma -> e- + 7 gamma, all 1024 states summed: the first points of\n")
        f.write("# k7_summed_oracle.txt with the brute-force FP64 oracle's |M|^2 and its\n")
        f.write("# dual-number gradient d|M|^2/d(px, py, pz) of the 7 outgoing photons (energies\n")
        f.write("# on shell), written by tests/golden/make_golden.py --grad.\n")
        f.write("# per point: one line m2, then 7 lines dpx dpy dpz (photons 1..7)\n")
        for i in range(n):
            f.write(f"{m2[i]:.17e}\n")
            for j in range(k):
                f.write(" ".join(f"{x:.17e}" for x in g[i, j]) + "\n")


def load_k7_grad():
    rows = [l.split() for l in open(K7_GRAD_FILE) if l.strip() and not l.startswith("#")]
    k = 7
    per = k + 1
    n = len(rows) // per
    m2 = np.array([float(rows[i * per][0]) for i in range(n)])
    g = np.array([[[float(x) for x in rows[i * per + 1 + j]] for j in range(k)] for i in range(n)])
    mom, _, kap = load_k7()
    return mom[:n], m2, g, kap[:n]


if __name__ == "__main__":
    if "--grad" in sys.argv:
        main_grad()
    else:
        main()
