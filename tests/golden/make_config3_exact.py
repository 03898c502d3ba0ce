"""Writes config3_exact.txt: the lowest 16 eigenvalues (with multiplicity) of the 3D QSE
workload's discrete operator (P = [I3, sqrt2 I3], K = L = 8, V = 3 sum_j (cos y_j + cos y_{j+3})).

The window, Lambda and V all factor over the three spatial dimensions, so the operator is a
Kronecker sum of three copies of the n = 2 problem P = [1, sqrt2], K = L = 8, V = 3 (cos y1 +
cos y2) (Sec. 3.1, Sec. 4.1); its spectrum is the set of triple sums of that 256-point
problem's eigenvalues. Calls only the oracle: dense Hermitian eigh of the assembled operator.

    python tests/golden/make_config3_exact.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2404_04507_gb300 import workloads as W  # noqa: E402


def main():
    P1 = np.array([[1.0, math.sqrt(2.0)]])
    m1, c1 = W.cosine_modes(2, 3.0)
    win = O.build_window(P1, (8,), (8,))
    e1 = O.eigen.dense_eigs(win, O.grid_coefficients(m1, c1, win.lens))[0]
    exact = O.eigen.kronecker_lowest([e1, e1, e1], 16)
    with open(os.path.join(HERE, "config3_exact.txt"), "w") as f:
        f.write("# lowest 16 eigenvalues of the 16^6 3D QSE operator (config 3), exact as a\n")
        f.write("# Kronecker sum of three 256-point problems; written by make_config3_exact.py\n")
        for v in exact:
            f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
