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
