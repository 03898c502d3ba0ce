"""Discretised Hamiltonian H~ = Lambda + F V F^{-1} as a direct spectral convolution.

Oracle; test infrastructure only. Sec. 4.1 (Eq. pseudospectral vector) defines
H~ U~ = Lambda U~ + F V F^{-1} U~ with F = T F* (Sec. 3.3, Eq. F). Because F^{-1} places
U~_k at grid frequency rho(k) and V multiplies pointwise on G_{K,L}, the product equals,
in exact arithmetic, a cyclic convolution on the K* grid:
    (F V F^{-1} U~)_k = sum_m Vg_m U~*_{(rho(k) - m) mod (2K.., 2L..)},
where Vg are the grid Fourier coefficients of V: every parent mode m is folded onto the
grid by the aliasing formula of App. C (Eq. d1 aliasing). No FFT is used here.

The preconditioner is Eq. precond, M = diag(h_ii / |H~ e_i|^2). Every column of the
circulant carries the same off-diagonal entries, so |H~ e_i|^2 = h_ii^2 + sum_{m!=0}|Vg_m|^2.
For potentials that are not non-negative the diagonal is shifted by sigma so that
V + sigma >= 1 (the shift leaves eigenvectors unchanged; see ``potential_shift``).
"""
from __future__ import annotations

import numpy as np

from .window import Window


def grid_coefficients(modes, coef, lens) -> np.ndarray:
    """Vg on the K* grid: fold each parent mode m onto m mod (2K.., 2L..) (aliasing)."""
    Vg = np.zeros(tuple(lens), dtype=np.complex128)
    modes = np.asarray(modes, dtype=np.int64).reshape(-1, len(lens))
    for m, c in zip(modes, np.asarray(coef, dtype=np.complex128)):
        idx = tuple(int(v) % int(s) for v, s in zip(m, lens))
        Vg[idx] += c
    return Vg


def _as_block(psi: np.ndarray):
    psi = np.asarray(psi, dtype=np.complex128)
    return (psi[:, None], True) if psi.ndim == 1 else (psi, False)


def apply_stencil(win: Window, Vg: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """H~ psi for psi in window order, (N,) or (N, nvec)."""
    X, vec = _as_block(psi)
    idx = tuple(win.kstar.T)
    shifts = [tuple(int(v) for v in m) for m in np.argwhere(Vg != 0)]
    out = np.empty_like(X)
    for c in range(X.shape[1]):
        G = np.zeros(win.lens, dtype=np.complex128)
        G[idx] = X[:, c]
        acc = np.zeros_like(G)
        for m in shifts:
            # np.roll: rolled[i] = G[i - m] along every axis (cyclic)
            acc += Vg[m] * np.roll(G, shift=m, axis=tuple(range(G.ndim)))
        out[:, c] = acc[idx] + win.lam * X[:, c]
    return out[:, 0] if vec else out


def dense_matrix(win: Window, Vg: np.ndarray) -> np.ndarray:
    """Assembled N x N matrix H~[i, j] = Lambda_i delta_ij + Vg[(k*_i - k*_j) mod]."""
    N = win.N
    if N > 6000:
        raise ValueError("dense assembly is for tiny windows only")
    diff = (win.kstar[:, None, :] - win.kstar[None, :, :]) % np.asarray(win.lens)[None, None, :]
    H = Vg[tuple(diff[..., a] for a in range(diff.shape[-1]))].astype(np.complex128)
    H[np.arange(N), np.arange(N)] += win.lam
    return H


def potential_shift(Vg: np.ndarray) -> float:
    """sigma = sum_{m!=0} |Vg_m| - Re Vg_0 + 1, so that V(y) + sigma >= 1 everywhere."""
    zero = (0,) * Vg.ndim
    off = np.abs(Vg).sum() - abs(Vg[zero])
    return float(off - Vg[zero].real + 1.0)


def precond_diag(win: Window, Vg: np.ndarray, sigma: float | None = None) -> np.ndarray:
    """M_kk = h / (h^2 + sum_{m!=0} |Vg_m|^2), h = Lambda_k + Vg_0 + sigma (Eq. precond)."""
    zero = (0,) * Vg.ndim
    sigma = potential_shift(Vg) if sigma is None else sigma
    off2 = float((np.abs(Vg) ** 2).sum() - abs(Vg[zero]) ** 2)
    h = win.lam + Vg[zero].real + sigma
    return h / (h * h + off2)
