"""Pins of the paper's example problems as stated in workloads.py (Sec. 4.2, Examples 4.1-4.3).

Each lifted potential, summed from its Fourier modes by the oracle, must equal the printed
parent function V(y) at random lifted points, and its restriction v(x) = V(P^T x) the printed
physical potential; each P must be the printed projection matrix. The accuracy studies run on
the GPU must list exactly the windows of the printed tables they are compared with.
"""
import math

import numpy as np

from oracle import transform as T
from paper_2404_04507_gb300 import workloads as W

RNG = np.random.default_rng(17)


def _check(pb, V, v, P):
    assert np.allclose(pb.P, P, rtol=0, atol=1e-15)
    y = RNG.uniform(-10, 10, size=(50, pb.n))
    assert np.max(np.abs(T.evaluate_parent(pb.modes, pb.coef, y) - V(y))) < 1e-12
    x = RNG.uniform(-20, 20, size=(50, pb.d))
    assert np.max(np.abs(T.evaluate_parent(pb.modes, pb.coef, x @ pb.P) - v(x))) < 1e-11


def test_example_41():
    v0, a = 2.5, (math.sqrt(5.0) - 1.0) / 2.0
    pb = W.example_41(v0, 5, 20)
    _check(pb,
           lambda y: v0 * (2 - np.cos(y[:, 0]) - np.cos(y[:, 1])),
           lambda x: v0 * (2 - np.cos(2 * np.pi * x[:, 0]) - np.cos(2 * np.pi * a * x[:, 0])),
           2 * np.pi * np.array([[1.0, a]]))


def test_example_42():
    for b, t in ((0.8, 0.2), (0.5, 0.25), (0.5, 0.2)):
        beta, theta = b * math.pi, t * math.pi
        pb = W.example_42(beta, theta, 6, 20)
        _check(pb,
               lambda y: 4 - (np.cos(y[:, 0]) + 2 * np.cos(y[:, 1]) + np.cos(y[:, 2])),
               lambda x: 4 - (np.cos(beta * x[:, 0]) + 2 * np.cos(beta * x[:, 1])
                              + np.cos(beta * x[:, 0] * math.cos(theta)
                                       + beta * x[:, 1] * math.sin(theta))),
               beta * np.array([[1.0, 0.0, math.cos(theta)], [0.0, 1.0, math.sin(theta)]]))


def test_example_43():
    beta, theta, a = math.pi, 0.2 * math.pi, (math.sqrt(5.0) - 1.0) / 2.0
    c, s = math.cos(theta), math.sin(theta)
    pb = W.example_43(beta, 5, 10)
    _check(pb,
           lambda y: 6 - np.sum(np.cos(y), axis=1),
           lambda x: 6 - (np.cos(beta * x[:, 0]) + np.cos(beta * x[:, 1]) + np.cos(beta * x[:, 2])
                          + np.cos(beta * x[:, 0] * c + beta * x[:, 1] * s)
                          + np.cos(-beta * x[:, 0] * s + beta * x[:, 1] * c)
                          + np.cos(beta * a * x[:, 2])),
           beta * np.array([[1.0, 0.0, 0.0, c, -s, 0.0],
                            [0.0, 1.0, 0.0, s, c, 0.0],
                            [0.0, 0.0, 1.0, 0.0, 0.0, a]]))


def test_accuracy_studies_cover_the_golden_tables():
    # the GPU studies run exactly the windows the printed tables list, against the references
    # the tables name (the library is built first: importing the package loads it)
    from paper_2404_04507_gb300 import build
    build.build()
    from paper_2404_04507_gb300 import accuracy as A
    from conftest import read_golden

    def keys(wins):
        return {(p.method, int(p.K[0]), int(p.L[0])) for p in wins}

    for study, golden, ref in ((A.ex41_v25(), "table2_ex41_errors.txt", ("pm", 640, 1024)),
                               (A.ex41_v3(), "table4_ex41_v3_errors.txt", ("iwfpm", 10, 4096)),
                               (A.ex42("I"), "table5_ex42_errors.txt", ("iwfpm", 10, 160))):
        wins, reference, d = study
        rows = {(r[0], int(r[1]), int(r[2])) for r in read_golden(golden)}
        assert rows == keys(wins), golden
        assert (reference.method, int(reference.K[0]), int(reference.L[0])) == ref
    wins, reference, d = A.ex41_v25(reference="iwfpm96")
    assert (reference.method, int(reference.K[0]), int(reference.L[0])) == ("iwfpm", 5, 96)
