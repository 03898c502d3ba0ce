"""Algorithm 1 of the paper: the transform F = T F* and its inverse (oracle only).

Sec. 3.3: the standard DFT F* on the grid G_{K,L} (Eq. standard discrete Fourier) gives
U~*_{k*} = <U, phi_{k*}>_{K,L} = (1/N) sum_l U(y_l) e^{-i k*.y_l} (Eq. new_inner_product),
and the index-shift transform T relabels it onto the window: U~_k = U~*_{rho(k)} (Eq. F).
Grid points are y_l = (pi l_I / K, pi l_II / L) (Eq. G_KL). Here numpy's FFT serves as the
library DFT; the pieces below are used to cross-check the convolution operator and to
test the aliasing formula (App. C), never by the product path.
"""
from __future__ import annotations

import numpy as np

from .window import Window


def grid_points(lens) -> list:
    """Per-axis coordinates y_j = 2 pi l_j / lens_j, l_j in [0, lens_j)."""
    return [2.0 * np.pi * np.arange(s) / s for s in lens]


def sample_parent(modes, coef, lens) -> np.ndarray:
    """U(y_l) = sum_m c_m exp(i m.y_l) on G_{K,L}, evaluated term by term."""
    ys = np.meshgrid(*grid_points(lens), indexing="ij")
    out = np.zeros(tuple(lens), dtype=np.complex128)
    for m, c in zip(np.asarray(modes), np.asarray(coef)):
        phase = sum(float(mj) * yj for mj, yj in zip(m, ys))
        out += c * np.exp(1j * phase)
    return out


def forward(win: Window, Ugrid: np.ndarray) -> np.ndarray:
    """U~ = F U = T F* U: grid samples -> window coefficients (Alg. 1, steps 2-6)."""
    Ustar = np.fft.fftn(Ugrid) / Ugrid.size
    return Ustar[tuple(win.kstar.T)]


def inverse(win: Window, Ut: np.ndarray) -> np.ndarray:
    """U(y_l) = sum_{k in K_{K,L}} U~_k e^{i k.y_l} = sum_{k*} U~*_{k*} e^{i k*.y_l}."""
    G = np.zeros(win.lens, dtype=np.complex128)
    G[tuple(win.kstar.T)] = Ut
    return np.fft.ifftn(G) * G.size


def apply_fft(win: Window, Vgrid: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """H~ psi = Lambda psi + F (V . F^{-1} psi) with a sampled real potential grid."""
    psi = np.asarray(psi, dtype=np.complex128)
    if psi.ndim == 2:
        return np.stack([apply_fft(win, Vgrid, psi[:, c]) for c in range(psi.shape[1])], 1)
    return win.lam * psi + forward(win, Vgrid * inverse(win, psi))


def evaluate_quasi(win: Window, Ut: np.ndarray, x: np.ndarray) -> np.ndarray:
    """u(x) = sum_k U~_k e^{i (P k).x} at physical points x (M, d) (Eq. int)."""
    Pk = win.k.astype(np.float64) @ win.P.T          # (N, d)
    return np.exp(1j * (np.asarray(x) @ Pk.T)) @ Ut


def evaluate_parent(modes, coef, y: np.ndarray) -> np.ndarray:
    """U(y) = sum_m c_m e^{i m.y} at lifted points y (M, n)."""
    return np.exp(1j * (np.asarray(y) @ np.asarray(modes, dtype=np.float64).T)) @ np.asarray(coef)


def normalise_field(u: np.ndarray, at: int | None = None):
    """u0 / u0(xi*) with xi* the first point of largest modulus, and that index (Sec. 4.2: the
    field is divided by its maximal modulus; the paper leaves the global phase free, and this
    reading fixes it by making the field real and positive at xi*). |u|^2 is formed as
    re*re + im*im with each step rounded, so that the choice of xi* is reproducible. A field
    that is zero everywhere is returned unchanged with index 0.

    `at` gives xi* instead of searching for it. Comparing two fields needs one common point:
    for an even potential H is real symmetric, u(-x) = conj(u(x)) and mirror points tie in
    modulus exactly, so fields normalised at different twins differ by a phase factor."""
    u = np.asarray(u, dtype=np.complex128)
    a = u.real * u.real + u.imag * u.imag
    i = int(np.argmax(a)) if at is None else int(at)
    if a[i] == 0.0:
        return u.copy(), (0 if at is None else i)
    return u / u[i], i


def density(u: np.ndarray) -> np.ndarray:
    """rho = |u0|^2 of a normalised field (Sec. 4.2)."""
    u = np.asarray(u, dtype=np.complex128)
    return u.real * u.real + u.imag * u.imag


def field_error(u: np.ndarray, u_ref: np.ndarray) -> float:
    """E_f = ||u0 - u0*||_inf over the grid, both fields normalised (Sec. 4.2)."""
    return float(np.max(np.abs(np.asarray(u) - np.asarray(u_ref)))) if len(u) else 0.0
