"""The oracle's C/OpenMP apply (oracle/capply.c) against the numpy oracle it restates.

Both write out the same direct spectral convolution (Sec. 4.1, Sec. 3.3, App. C); the numpy
one is pinned by the other oracle tests (V = 0, Mathieu, Kronecker sums, Algorithm 1 via
FFT, Hermiticity). Same modes in the same order, so the two agree to the last bit here.
"""
import numpy as np
import pytest

import oracle as O
from oracle import capply
from paper_2404_04507_gb300 import workloads as W


@pytest.mark.parametrize("pb", [
    W.config_1d(),
    W.config_moire(eps=5.0, K=4, L=3),
    W.config_moire(eps=0.5, K=3, L=2, method="pm"),
    W.config_3d(K=2, L=2),
    W.example_41(2.5, 5, 20),
    W.example_42(0.8 * np.pi, 0.2 * np.pi, 3, 6),
    W.example_43(1.0, 2, 2),
], ids=lambda p: p.name)
def test_c_apply_equals_numpy_oracle(pb):
    win = O.build_window(pb.P, pb.K, pb.L, method=pb.method)
    Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
    X = W.random_block(win.N, 3, seed=11)
    want = O.apply_stencil(win, Vg, X)
    got = capply.apply(win, Vg, X)
    assert np.max(np.abs(got - want)) <= 1e-15 * np.max(np.abs(want))
    assert np.allclose(capply.apply(win, Vg, X[:, 1]), want[:, 1], rtol=0, atol=1e-13)


def test_c_apply_is_hermitian():
    pb = W.config_moire(eps=2.0, K=3, L=3)
    win = O.build_window(pb.P, pb.K, pb.L)
    Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
    X = W.random_block(win.N, 2, seed=3)
    HX = capply.apply(win, Vg, X)
    a = np.vdot(X[:, 0], HX[:, 1])
    b = np.vdot(HX[:, 0], X[:, 1])
    assert abs(a - b) <= 1e-13 * abs(a)
