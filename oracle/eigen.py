"""Reference eigenpairs and spectral quantities of H~ (oracle; test infrastructure only).

Sec. 4.1 asks for the lowest eigenpairs of H~ U~ = E U~. The oracle computes them by
library eigensolvers applied to the oracle's own operator: dense Hermitian ``eigh`` on
the assembled matrix for tiny windows, Lanczos (``eigsh``) or scipy's LOBPCG with the
diagonal preconditioner of Eq. precond for larger ones. ``condition_number`` gives
lambda_max / lambda_min of H~ or of M^{1/2} H~ M^{1/2} (the reading of "condition number
of M H~" for Table 1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .operator import apply_stencil, dense_matrix, precond_diag
from .window import Window


def dense_eigs(win: Window, Vg: np.ndarray, nev: int | None = None):
    w, v = np.linalg.eigh(dense_matrix(win, Vg))
    nev = win.N if nev is None else nev
    return w[:nev], v[:, :nev]


def linear_operator(win: Window, Vg: np.ndarray, scale: np.ndarray | None = None):
    """H~ (or D H~ D for a positive diagonal D = ``scale``) as a scipy LinearOperator."""
    def mv(x):
        x = np.asarray(x, dtype=np.complex128).reshape(win.N, -1)
        if scale is None:
            return apply_stencil(win, Vg, x)
        return scale[:, None] * apply_stencil(win, Vg, scale[:, None] * x)
    return spla.LinearOperator((win.N, win.N), matvec=mv, matmat=mv, dtype=np.complex128)


def lowest_eigs(win: Window, Vg: np.ndarray, nev: int, tol: float = 1e-12, seed: int = 0):
    """Lowest nev eigenpairs by Lanczos on the oracle operator (ascending)."""
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(win.N) + 1j * rng.standard_normal(win.N)
    w, v = spla.eigsh(linear_operator(win, Vg), k=nev, which="SA", tol=tol, v0=v0,
                      ncv=max(4 * nev, 40))
    order = np.argsort(w)
    return w[order], v[:, order]


def _extreme(op, N, which, tol, seed, precond=None, maxiter=60):
    rng = np.random.default_rng(seed)
    if precond is None:
        v0 = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        w = spla.eigsh(op, k=1, which=which, tol=tol, v0=v0, ncv=16,
                       return_eigenvectors=False)
        return float(w[0])
    X = rng.standard_normal((N, 2)) + 1j * rng.standard_normal((N, 2))
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", UserWarning)
        w, _ = spla.lobpcg(op, X, M=precond, largest=(which == "LA"), tol=tol,
                           maxiter=maxiter)
    return float(np.min(w) if which == "SA" else np.max(w))


def condition_number(win: Window, Vg: np.ndarray, preconditioned: bool,
                     tol: float = 1e-4, seed: int = 0) -> float:
    """lambda_max / lambda_min of H~, or of M^{1/2} H~ M^{1/2} when preconditioned.

    Tolerances aim at four significant digits (Table 1 prints three). The low end of
    H~ is found by preconditioned LOBPCG (M of Eq. precond), where the residual-based
    eigenvalue error is quadratic in the residual.
    """
    m = precond_diag(win, Vg, sigma=0.0)
    if preconditioned:
        s = np.sqrt(m)
        op = linear_operator(win, Vg, scale=s)
        lo = _extreme(op, win.N, "SA", tol, seed)
        hi = _extreme(op, win.N, "LA", tol, seed + 1)
        return hi / lo
    op = linear_operator(win, Vg)
    pre = spla.LinearOperator((win.N, win.N), dtype=np.complex128,
                              matvec=lambda x: m * np.asarray(x).reshape(-1),
                              matmat=lambda x: m[:, None] * np.asarray(x))
    lo = _extreme(op, win.N, "SA", 1e-6, seed, precond=pre)
    hi = _extreme(op, win.N, "LA", tol, seed + 1)
    return hi / lo


def residual_norms(win: Window, Vg: np.ndarray, X: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """|H~ x_i - lambda_i x_i|_2 / |x_i|_2 with the oracle operator (FP64)."""
    X = np.asarray(X, dtype=np.complex128)
    R = apply_stencil(win, Vg, X) - X * np.asarray(lam)[None, :]
    return np.linalg.norm(R, axis=0) / np.linalg.norm(X, axis=0)


def kronecker_lowest(parts_eigs, nev: int) -> np.ndarray:
    """Lowest nev sums lambda_a + lambda_b + ... over independent blocks (with multiplicity)."""
    acc = np.array([0.0])
    for w in parts_eigs:
        acc = np.sort((acc[:, None] + np.asarray(w)[None, :]).ravel())[: max(nev, 1) * 8]
    return acc[:nev]
