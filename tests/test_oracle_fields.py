"""Pins of the oracle's physical-space field metrics (Sec. 4.2: u0 on a uniform grid,
normalised by its maximal modulus, rho = |u0|^2 and E_f = ||u0 - u0*||_inf).

The normalisation's phase is a reading (the paper leaves it free): the field is divided by
its value at the first point of largest modulus. The pins are hand-worked examples, the
invariance under any nonzero complex scale, and a two-mode field on the paper's 1D grid
whose maximum and normalised values follow in closed form.
"""
import math

import numpy as np

import oracle as O
from oracle import transform as T
from paper_2404_04507_gb300 import workloads as W


def test_normalise_hand_example():
    u, i = T.normalise_field(np.array([1.0, -2.0, 1j]))
    assert i == 1
    assert np.array_equal(u, np.array([-0.5, 1.0, -0.5j]))
    assert np.array_equal(T.density(u), np.array([0.25, 1.0, 0.25]))


def test_normalise_at_a_given_point():
    u, i = T.normalise_field(np.array([1.0, -2.0, 1j]), at=2)
    assert i == 2
    assert np.array_equal(u, np.array([-1j, 2j, 1.0]))


def test_mirror_twins_of_an_even_potential():
    # V even and real: H~ is real symmetric in the k basis, so the ground state's coefficients
    # are real up to one phase and u(-x) = conj(u(x)): |u| ties exactly at mirror points, and
    # normalising at the two twins gives fields that differ by the phase factor u(x)/conj(u(x))
    pb = W.config_1d(K=6, L=8, eps=3.0)
    win = O.build_window(pb.P, pb.K, pb.L)
    V = O.eigen.dense_eigs(win, O.grid_coefficients(pb.modes, pb.coef, win.lens), 1)[1][:, 0]
    x = np.array([[-37.3], [37.3]])
    u = T.evaluate_quasi(win, V, x)
    assert abs(u[1] - np.conj(u[0])) <= 1e-13 * abs(u[0])
    a, _ = T.normalise_field(u, at=0)
    b, _ = T.normalise_field(u, at=1)
    assert abs(T.field_error(a, b) - abs(u[0] / u[1] - 1) * abs(b[0])) <= 1e-13


def test_normalise_ties_take_the_first_point():
    u, i = T.normalise_field(np.array([0.5, 2.0, -2.0, 2j]))
    assert i == 1
    assert np.array_equal(u, np.array([0.25, 1.0, -1.0, 1j]))


def test_normalise_removes_scale_and_phase():
    rng = np.random.default_rng(7)
    u = rng.standard_normal(500) + 1j * rng.standard_normal(500)
    a, i = T.normalise_field(u)
    b, j = T.normalise_field(3.5 * np.exp(0.7j) * u)
    assert i == j
    assert abs(a[i] - 1.0) <= 1e-15 and np.max(np.abs(a)) <= 1.0 + 1e-15
    assert T.field_error(a, b) <= 4e-15


def test_zero_field_is_unchanged():
    u, i = T.normalise_field(np.zeros(4, dtype=complex))
    assert i == 0 and not np.any(u)


def test_field_error_closed_form():
    assert T.field_error(np.array([1.0, 0.5]), np.array([1.0, 0.5 + 1e-3j])) == 1e-3
    assert T.field_error(np.array([1.0, -1.0]), np.array([-1.0, 1.0])) == 2.0
    assert T.field_error(np.array([]), np.array([])) == 0.0


def test_physical_grid_of_the_paper():
    for d, cnt in ((1, 10001), (2, 1001), (3, 101)):
        g = W.physical_grid(d)
        half = 5.0 * 10.0 ** (3 - d)
        assert g.shape == (cnt ** d, d)
        assert g[0, 0] == -half and abs(g[-1, 0] - half) < 1e-9
        assert abs(g[1, -1] - g[0, -1] - 0.1) < 1e-12


def test_two_mode_field_on_the_1d_grid():
    # u(x) = e^{i x} + e^{i sqrt5 x} from the window coefficients at k = (1, 0) and (0, 1):
    # |u|^2 = 2 + 2 cos((sqrt5 - 1) x) peaks only at x = 0 on the grid (value 4), so the
    # normalised field is u / 2 and rho = (1 + cos((sqrt5 - 1) x)) / 2
    pb = W.config_1d(K=4, L=4)
    win = O.build_window(pb.P, pb.K, pb.L)
    c = np.zeros(win.N, dtype=complex)
    for kv in ((1, 0), (0, 1)):
        c[np.all(win.k == np.array(kv), axis=1)] = 1.0
    x = W.physical_grid(1)
    u, i = T.normalise_field(T.evaluate_quasi(win, c, x))
    assert i == 5000 and x[i, 0] == 0.0
    xs = x[:, 0]
    assert np.max(np.abs(u - (np.exp(1j * xs) + np.exp(1j * math.sqrt(5.0) * xs)) / 2)) < 1e-12
    rho = T.density(u)
    assert np.max(np.abs(rho - (1 + np.cos((math.sqrt(5.0) - 1) * xs)) / 2)) < 1e-12


def test_grid_descriptor_names_the_observation_grid():
    # the (origin, step, count) handed to the separable grid evaluation expands, with the
    # kernel's own rounding (origin + index * step), to exactly the observation grid's points
    for rows in (None, 8):
        (o0, o1), (h0, h1), (c0, c1) = W.grid_descriptor(2, rows)
        pts = W.physical_grid(2, rows=rows)
        x0 = o0 + np.arange(c0) * h0
        x1 = o1 + np.arange(c1) * h1
        mesh = np.stack(np.meshgrid(x0, x1, indexing="ij"), -1).reshape(-1, 2)
        assert mesh.shape == pts.shape and np.array_equal(mesh, pts)
