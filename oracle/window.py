"""Irrational window, index-shift map and kinetic diagonal (oracle; test infrastructure only).

Follows the paper's Sec. 3.1 (window W_{K,L}, index set K_{K,L} = W cap Z^n, Eq. non-tensor),
Sec. 3.2 (index-shift map rho, Eq. index mod; its inverse in two steps, Eqs. inverse1-3)
and Sec. 4.1 (Lambda = 1/2 diag(|Pk|^2), Eq. discrete_Lambda).

Readings where the paper leaves a choice open:
  * the shift is either the exact one of Eq. inverse3 (q = (Q k_II)_j) or the rounded one
    (q replaced by round-half-away-from-zero(q)); the rounded one is the only one that
    reproduces the printed condition numbers of Table 1;
  * q = Q k_II is summed left to right with every product and sum rounded separately
    (no fused multiply-add), so that another implementation can classify identically;
  * a shifted bound that lies within 1e-9 of an integer (or, rounded, of a half-integer)
    without being one is ambiguous in floating point and raises ``WindowTie``;
  * the projection method (PM) is the same construction with the shear switched off
    (Q = 0): the box [-K,K)^d x [-L,L)^{n-d} of Sec. 2.
Window order (the storage order of a coefficient vector): k_II lexicographic (slowest),
then k_I lexicographic; every k_I slice is a run of 2K_j consecutive integers per axis.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

TIE_EPS = 1e-9


class WindowTie(ValueError):
    """A window bound is too close to an integer to be classified reliably."""


def split_Q(P: np.ndarray) -> np.ndarray:
    """Q = P_I^{-1} P_II (Sec. 3.1) by a library linear solve."""
    P = np.asarray(P, dtype=np.float64)
    d = P.shape[0]
    PI, PII = P[:, :d], P[:, d:]
    if np.linalg.cond(PI) > 1e12:
        raise ValueError("P_I is singular or ill-conditioned; reorder the columns of P")
    if d == 1:
        return PII / PI[0, 0]
    return np.linalg.solve(PI, PII)


def _q_fixed_order(Q: np.ndarray, kII: np.ndarray) -> np.ndarray:
    """q_j = sum_i Q[j,i] kII[:,i], left to right, separately rounded products and sums."""
    M = kII.shape[0]
    d = Q.shape[0]
    q = np.zeros((M, d), dtype=np.float64)
    for j in range(d):
        acc = np.zeros(M, dtype=np.float64)
        for i in range(Q.shape[1]):
            prod = np.multiply(Q[j, i], kII[:, i].astype(np.float64))
            acc = np.add(acc, prod) if i else prod
        q[:, j] = acc
    return q


def _round_half_away(q: np.ndarray) -> np.ndarray:
    r = np.trunc(q)
    f = q - r
    return r + np.where(np.abs(f) >= 0.5, np.sign(q), 0.0)


def _check_ties(K: np.ndarray, q: np.ndarray, shift_round: bool) -> None:
    if shift_round:
        h = q - np.floor(q) - 0.5
        bad = (np.abs(h) < TIE_EPS) & (h != 0.0)
    else:
        t = -K[None, :] - q
        dist = np.abs(t - np.round(t))
        bad = (dist < TIE_EPS) & (dist != 0.0)
    if np.any(bad):
        raise WindowTie("window bound within 1e-9 of an integer")


def _shift(q: np.ndarray, shift_round: bool) -> np.ndarray:
    return _round_half_away(q) if shift_round else q


@dataclass
class Window:
    P: np.ndarray
    K: np.ndarray
    L: np.ndarray
    Q: np.ndarray
    lens: tuple            # (2K_1..2K_d, 2L_1..2L_{n-d}), the K* grid sides
    k: np.ndarray          # (N, n) true indices, window order
    kstar: np.ndarray      # (N, n) rho(k)
    lam: np.ndarray        # (N,) 1/2 |P k|^2

    @property
    def N(self) -> int:
        return int(self.k.shape[0])

    @property
    def d(self) -> int:
        return int(self.P.shape[0])

    @property
    def n(self) -> int:
        return int(self.P.shape[1])


def kinetic(P: np.ndarray, k: np.ndarray) -> np.ndarray:
    """Lambda_k = 1/2 |P k|^2 on the true index k (Eq. discrete_Lambda)."""
    Pk = np.zeros((k.shape[0], P.shape[0]), dtype=np.float64)
    for a in range(P.shape[0]):
        for j in range(P.shape[1]):
            Pk[:, a] += P[a, j] * k[:, j]
    return 0.5 * np.sum(Pk * Pk, axis=1)


def build_window(P, K, L, shift_round: bool = False, method: str = "iwfpm") -> Window:
    """K_{K,L} through the paper's explicit two-step inverse of rho (Eqs. inverse1-3)."""
    P = np.asarray(P, dtype=np.float64)
    d, n = P.shape
    K = np.asarray(K, dtype=np.int64).reshape(d)
    L = np.asarray(L, dtype=np.int64).reshape(n - d)
    Q = np.zeros((d, n - d)) if method == "pm" else split_Q(P)
    lens = tuple(int(2 * v) for v in K) + tuple(int(2 * v) for v in L)
    # every k* of the hyperrectangle K*_{K,L} = [0,2K)^d x [0,2L)^{n-d}
    kstar = np.array(list(itertools.product(*[range(m) for m in lens])), dtype=np.int64)
    # step 1 (Eq. inverse2): k_II from k*_II
    ksII = kstar[:, d:]
    kII = np.where(ksII < L[None, :], ksII, ksII - 2 * L[None, :])
    q = _q_fixed_order(Q, kII)
    _check_ties(K, q, shift_round)
    s = _shift(q, shift_round)
    # step 2 (Eq. inverse3): R_j = ceil((-K - q_j) / 2K) 2K, then one of two cases
    twoK = 2 * K[None, :]
    R = np.ceil((-K[None, :] - s) / twoK) * twoK
    ksI = kstar[:, :d].astype(np.float64)
    first = (ksI + R) + s < K[None, :]
    kI = np.where(first, ksI + R, ksI + R - twoK).astype(np.int64)
    k = np.concatenate([kI, kII], axis=1)
    # window order: k_II lexicographic, then k_I lexicographic
    keys = [k[:, j] for j in range(d - 1, -1, -1)] + [k[:, j] for j in range(n - 1, d - 1, -1)]
    order = np.lexsort(keys)
    k = k[order]
    kstar = kstar[order]
    return Window(P, K, L, Q, lens, k, kstar, kinetic(P, k))


def brute_force_window(P, K, L, shift_round: bool = False, method: str = "iwfpm") -> np.ndarray:
    """Z^n cap W_{K,L} by enumerating a bounding box (Sec. 3.1 definition), window order."""
    P = np.asarray(P, dtype=np.float64)
    d, n = P.shape
    K = np.asarray(K, dtype=np.int64).reshape(d)
    L = np.asarray(L, dtype=np.int64).reshape(n - d)
    Q = np.zeros((d, n - d)) if method == "pm" else split_Q(P)
    kII = np.array(list(itertools.product(*[range(-l, l) for l in L])), dtype=np.int64)
    kII = kII.reshape(-1, n - d)
    q = _q_fixed_order(Q, kII)
    s = _shift(q, shift_round)
    span = int(np.ceil(np.max(np.abs(s)))) + 1 if s.size else 1
    out = []
    for r in range(kII.shape[0]):
        ranges = [range(-int(K[j]) - span - 1, int(K[j]) + span + 2) for j in range(d)]
        for kI in itertools.product(*ranges):
            v = np.asarray(kI, dtype=np.float64) + s[r]
            if np.all(v >= -K) and np.all(v < K):
                out.append(list(kI) + list(kII[r]))
    return np.asarray(out, dtype=np.int64)
