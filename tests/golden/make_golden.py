"""Writes tests/golden/hex37_oracle.txt by calling only the oracle and the input generators.

The fixture pins the oracle against accidental change and checks that the x86
and Arm builds agree: visibilities of the 37-antenna hexagon (Gaussian beam,
FWHM 10 deg at 150 MHz, one channel, one time) for 40 seeded point sources, by
the FP64 direct sum of Eq. (1) under the point-source approximation (Eq. 3).
Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle.oracle import OracleProblem, oracle_vis          # noqa: E402
from paper_2506_02130_gb300 import workloads as W          # noqa: E402


def main():
    prob = W.config_small(seed=11, n_src=40)
    pairs = prob.pairs[::17]
    v = oracle_vis(OracleProblem.from_workload(prob, pairs=pairs), "literal")[0, 0, :, 0]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hex37_oracle.txt")
    with open(out, "w") as f:
        f.write("# oracle direct sum (Eq. 1, Eq. 3): config_small(seed=11, n_src=40), pairs[::17]\n")
        f.write("# i j re im\n")
        for (i, j), z in zip(pairs, v):
            f.write(f"{i} {j} {z.real:.17e} {z.imag:.17e}\n")


if __name__ == "__main__":
    main()
