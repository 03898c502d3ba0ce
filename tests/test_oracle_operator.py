"""Pins of the oracle's discrete Hamiltonian H~ = Lambda + F V F^{-1} (Sec. 3.3, 4.1, App. C).

Each test ties the oracle to something other than itself: closed forms, a textbook
special case (Mathieu), a library FFT route through Algorithm 1, brute-force evaluation of
the quasiperiodic function, the aliasing formula, separability and exact symmetries.
"""
import math

import numpy as np
import pytest
from scipy.special import mathieu_a

import oracle as O
from oracle import transform as T
from paper_2404_04507_gb300 import workloads as W


def _rand(N, seed, nvec=None):
    rng = np.random.default_rng(seed)
    shape = (N,) if nvec is None else (N, nvec)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


SMALL = [
    (np.array([[1.0, math.sqrt(5.0)]]), [3], [4]),
    (W.moire_P(math.pi / 6), [2, 2], [2, 2]),
    (W.random_P(2, 3, seed=3), [3, 2], [2]),
    (np.concatenate([np.eye(3), math.sqrt(2) * np.eye(3)], 1), [1, 1, 1], [1, 1, 2]),
]


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_hermitian(case):
    P, K, L = SMALL[case]
    win = O.build_window(P, K, L)
    m, c = W.random_modes(win.n, 4, 2, seed=case)
    Vg = O.grid_coefficients(m, c, win.lens)
    x, y = _rand(win.N, 1), _rand(win.N, 2)
    lhs = np.vdot(x, O.apply_stencil(win, Vg, y))
    rhs = np.vdot(O.apply_stencil(win, Vg, x), y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    H = O.dense_matrix(win, Vg)
    assert np.allclose(H, H.conj().T, atol=1e-14)


@pytest.mark.parametrize("case", range(len(SMALL)))
def test_free_particle_spectrum_is_kinetic(case):
    # V = 0: eigenvalues are exactly { |P k|^2 / 2 : k in K_{K,L} } (closed form)
    P, K, L = SMALL[case]
    win = O.build_window(P, K, L)
    brute = O.brute_force_window(P, K, L)
    closed = np.sort(0.5 * np.sum((brute.astype(float) @ P.T) ** 2, axis=1))
    Vg = np.zeros(win.lens, dtype=complex)
    w, _ = O.eigen.dense_eigs(win, Vg)
    assert np.allclose(w, closed, rtol=1e-13, atol=1e-13)


def test_constant_potential_shifts_spectrum():
    P, K, L = SMALL[1]
    win = O.build_window(P, K, L)
    Vg = O.grid_coefficients(np.zeros((1, 4), int), np.array([2.75 + 0j]), win.lens)
    w, _ = O.eigen.dense_eigs(win, Vg)
    assert np.allclose(w, np.sort(win.lam) + 2.75, rtol=1e-13)


@pytest.mark.parametrize("case", range(len(SMALL)))
@pytest.mark.parametrize("radius", [1, 3])
def test_convolution_equals_algorithm1_fft_route(case, radius):
    # radius 3 puts modes outside the grid's Nyquist range: aliasing must agree too
    P, K, L = SMALL[case]
    win = O.build_window(P, K, L)
    m, c = W.random_modes(win.n, 4, radius, seed=10 + case)
    Vg = O.grid_coefficients(m, c, win.lens)
    Vgrid = T.sample_parent(m, c, win.lens)
    assert np.max(np.abs(Vgrid.imag)) < 1e-12
    X = _rand(win.N, 5, nvec=3)
    a = O.apply_stencil(win, Vg, X)
    b = T.apply_fft(win, Vgrid.real, X)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_interpolation_is_exact_for_band_limited_parents():
    # App. C, Eq. d1 aliasing: modes inside K_{K,L} come back unchanged at their true index
    P = W.moire_P(math.pi / 6)
    win = O.build_window(P, [3, 3], [2, 2])
    rng = np.random.default_rng(0)
    pick = rng.choice(win.N, size=12, replace=False)
    modes, coef = win.k[pick], rng.standard_normal(12) + 1j * rng.standard_normal(12)
    Ut = T.forward(win, T.sample_parent(modes, coef, win.lens))
    expect = np.zeros(win.N, dtype=complex)
    expect[pick] = coef
    assert np.max(np.abs(Ut - expect)) < 1e-14


def test_aliasing_formula_for_modes_outside_window():
    P = np.array([[1.0, math.sqrt(5.0)]])
    win = O.build_window(P, [2], [3])
    m = np.array([[7, 1], [-9, -8], [0, 13]])      # all outside K_{K,L}
    c = np.array([1.0 + 0.5j, -0.25j, 2.0])
    Ut = T.forward(win, T.sample_parent(m, c, win.lens))
    expect = np.zeros(win.N, dtype=complex)
    for mv, cv in zip(m, c):
        # the unique window index congruent to m modulo (2K, 2L) receives c
        hit = np.all(np.mod(win.k - mv, np.asarray(win.lens)) == 0, axis=1)
        assert hit.sum() == 1
        expect[hit] += cv
    assert np.max(np.abs(Ut - expect)) < 1e-14


def test_quasiperiodic_evaluation_matches_parent_on_projection():
    # u(x) = sum_k U~_k e^{i Pk.x} equals U(P^T x) for a band-limited parent (Eq. int)
    P = W.moire_P(math.pi / 6)
    win = O.build_window(P, [3, 3], [2, 2])
    rng = np.random.default_rng(4)
    pick = rng.choice(win.N, size=9, replace=False)
    modes, coef = win.k[pick], rng.standard_normal(9) + 1j * rng.standard_normal(9)
    Ut = T.forward(win, T.sample_parent(modes, coef, win.lens))
    x = rng.uniform(-20, 20, size=(25, 2))
    assert np.allclose(T.evaluate_quasi(win, Ut, x),
                       T.evaluate_parent(modes, coef, x @ P), atol=1e-11)


def test_parseval():
    win = O.build_window(W.random_P(2, 4, seed=1), [2, 3], [2, 1])
    Ut = _rand(win.N, 8)
    U = T.inverse(win, Ut)
    assert np.sum(np.abs(U) ** 2) / U.size == pytest.approx(np.sum(np.abs(Ut) ** 2), rel=1e-13)


@pytest.mark.parametrize("v0", [0.5, 2.0, 5.0])
def test_mathieu_special_case(v0):
    # Q = 0 (P = [1, 0]) decouples the k_II slices; each is -u''/2 + v0(1 - cos y) u = E u,
    # i.e. Mathieu's equation with a = 8(E - v0), q = 4 v0: E0 = v0 + a_0(4 v0) / 8.
    P = np.array([[1.0, 0.0]])
    m, c = W.cosine_modes(2, -v0, const=v0, axes=[0])
    win = O.build_window(P, [16], [2])
    Vg = O.grid_coefficients(m, c, win.lens)
    w, _ = O.eigen.dense_eigs(win, Vg, nev=8)
    e0 = v0 + mathieu_a(0, 4.0 * v0) / 8.0
    assert np.allclose(w[:4], e0, rtol=1e-8, atol=1e-9)       # 2L-fold degenerate
    assert w[4] > e0 + 1e-3


def test_kronecker_sum_of_separable_problem():
    a, b, eps, K, L = math.sqrt(2.0), math.sqrt(3.0), 1.3, 3, 2
    P = np.array([[1.0, 0.0, a, 0.0], [0.0, 1.0, 0.0, b]])
    m, c = W.cosine_modes(4, eps)
    win = O.build_window(P, [K, K], [L, L])
    w, _ = O.eigen.dense_eigs(win, O.grid_coefficients(m, c, win.lens), nev=20)
    parts = []
    for coeff in (a, b):
        Pp = np.array([[1.0, coeff]])
        mp, cp = W.cosine_modes(2, eps)
        wp = O.build_window(Pp, [K], [L])
        parts.append(O.eigen.dense_eigs(wp, O.grid_coefficients(mp, cp, wp.lens))[0])
    assert np.allclose(w, O.eigen.kronecker_lowest(parts, 20), rtol=1e-12, atol=1e-12)


def test_grid_lattice_phases_leave_spectrum_invariant():
    P = W.moire_P(math.pi / 6)
    K = L = 2
    win = O.build_window(P, [K, K], [L, L])
    m0, c0 = W.cosine_modes(4, 0.8)
    phases = np.array([math.pi / K, 3 * math.pi / K, -math.pi / L, 2 * math.pi / L])
    m1, c1 = W.cosine_modes(4, 0.8, phases)
    w0, _ = O.eigen.dense_eigs(win, O.grid_coefficients(m0, c0, win.lens), nev=30)
    w1, _ = O.eigen.dense_eigs(win, O.grid_coefficients(m1, c1, win.lens), nev=30)
    assert np.allclose(w0, w1, rtol=1e-12, atol=1e-12)


def test_preconditioner_closed_form_matches_definition():
    # Eq. precond: M_ii = h_ii / |H~ e_i|^2 (non-negative potential, no shift)
    win = O.build_window(np.array([[1.0, math.sqrt(5.0)]]), [4], [5])
    m, c = W.cosine_modes(2, -1.5, const=3.0)
    Vg = O.grid_coefficients(m, c, win.lens)
    H = O.dense_matrix(win, Vg)
    direct = np.real(np.diag(H)) / np.sum(np.abs(H) ** 2, axis=0)
    assert np.allclose(O.precond_diag(win, Vg, sigma=0.0), direct, rtol=1e-14)


def test_potential_shift_makes_diagonal_positive():
    m, c = W.cosine_modes(4, 5.0)
    win = O.build_window(W.moire_P(math.pi / 6), [2, 2], [2, 2])
    Vg = O.grid_coefficients(m, c, win.lens)
    sigma = O.potential_shift(Vg)
    assert sigma == pytest.approx(4 * 5.0 + 1.0)
    assert np.all(O.precond_diag(win, Vg) > 0)


def test_lanczos_route_matches_dense():
    win = O.build_window(W.moire_P(math.pi / 6), [2, 3], [2, 2])
    m, c = W.cosine_modes(4, 2.0)
    Vg = O.grid_coefficients(m, c, win.lens)
    wd, _ = O.eigen.dense_eigs(win, Vg, nev=6)
    wl, X = O.eigen.lowest_eigs(win, Vg, 6)
    assert np.allclose(wl, wd, rtol=1e-10, atol=1e-10)
    assert np.max(O.eigen.residual_norms(win, Vg, X, wl)) < 1e-8
