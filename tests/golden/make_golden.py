"""Writes the stored oracle values used by the GPU tests whose oracle cost is
too high to recompute in a test run (k = 7, all 1024 states summed: about
8e10 FLOP per point).  Calls only the oracle and the seeded input generator.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2511_19456_b300 import phasespace as ps  # noqa: E402

K7_FILE = os.path.join(HERE, "k7_summed_oracle.txt")


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


if __name__ == "__main__":
    main()
