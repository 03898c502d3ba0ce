"""Seeded synthetic problem generators shared by the tests, the benchmark and the oracle.

This module only *states* problems: projection matrices, window sizes, potential Fourier
modes and random start blocks. It contains none of the method's arithmetic (no window,
no index shift, no transform, no operator), so the CUDA path and the CPU oracle can both
draw their inputs from here without sharing any computation.

Problem conventions (the paper's notation, Sec. 2 and Sec. 4.1):
  * ``P`` is the d x n projection matrix, u(x) = U(P^T x).
  * ``K`` (length d) and ``L`` (length n-d) size the irrational window W_{K,L} (Sec. 3.1);
    for the projection method (PM) they size the box [-K,K)^d x [-L,L)^{n-d}.
  * the lifted potential is V(y) = sum_m c_m exp(i m.y); a real V comes as +-m pairs with
    conjugate coefficients. ``modes`` is an int array (nmodes, n), ``coef`` complex (nmodes,).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = (1.0 + math.sqrt(5.0)) / 2.0          # (1+sqrt5)/2, worked window example (Fig. 1)
ALPHA_EX41 = (math.sqrt(5.0) - 1.0) / 2.0       # alpha of Example 4.1


@dataclass
class Problem:
    name: str
    P: np.ndarray                  # (d, n) float64
    K: tuple                       # d ints
    L: tuple                       # n-d ints
    modes: np.ndarray              # (nmodes, n) int64
    coef: np.ndarray               # (nmodes,) complex128
    nev: int = 1
    block: int = 1
    precision: str = "f64"         # "f64" or "c64" (complex64 apply, float64 solve)
    method: str = "iwfpm"          # "iwfpm" or "pm"
    shift_round: bool = False      # False: exact ceil shift; True: rounded shift
    meta: dict = field(default_factory=dict)

    @property
    def d(self) -> int:
        return int(self.P.shape[0])

    @property
    def n(self) -> int:
        return int(self.P.shape[1])

    @property
    def dof(self) -> int:
        out = 1
        for k in self.K:
            out *= 2 * int(k)
        for l in self.L:
            out *= 2 * int(l)
        return out


def cosine_modes(n: int, eps, phases=None, const: float = 0.0, axes=None):
    """Modes of V(y) = const + sum_j eps_j cos(y_j + phi_j) over the listed lifted axes."""
    axes = list(range(n)) if axes is None else list(axes)
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (len(axes),))
    phases = np.zeros(len(axes)) if phases is None else np.asarray(phases, dtype=np.float64)
    modes, coef = [], []
    if const != 0.0:
        modes.append([0] * n)
        coef.append(complex(const))
    for a, e, ph in zip(axes, eps, phases):
        m = [0] * n
        m[a] = 1
        modes.append(list(m))
        coef.append(0.5 * e * complex(math.cos(ph), math.sin(ph)))
        m[a] = -1
        modes.append(list(m))
        coef.append(0.5 * e * complex(math.cos(ph), -math.sin(ph)))
    return np.asarray(modes, dtype=np.int64).reshape(-1, n), np.asarray(coef, dtype=np.complex128)


def moire_P(theta: float) -> np.ndarray:
    """P = [I_2, R_theta]: columns e1, e2, R e1, R e2 (twisted square lattices).

    At theta = pi/6 the entries are stated exactly (cos = sqrt3/2, sin = 1/2): the float
    value of sin(pi/6) is 0.49999999999999994, which would turn the window's exact
    rational ties into near-ties.
    """
    if abs(theta - math.pi / 6) < 1e-15:
        c, s = math.sqrt(3.0) / 2.0, 0.5
    else:
        c, s = math.cos(theta), math.sin(theta)
    return np.array([[1.0, 0.0, c, -s], [0.0, 1.0, s, c]], dtype=np.float64)


def config_1d(K: int = 12, L: int = 16, eps: float = 1.0, method: str = "iwfpm") -> Problem:
    """1D QSE V(x)=eps(cos x + cos sqrt5 x), P=[1, sqrt5], n=2, 8 eigenpairs, FP64."""
    P = np.array([[1.0, math.sqrt(5.0)]])
    m, c = cosine_modes(2, eps)
    return Problem("qse1d", P, (K,), (L,), m, c, nev=8, block=8, method=method)


def config_moire(eps: float = 0.5, K: int = 16, L: int = 16, theta: float = math.pi / 6,
                 method: str = "iwfpm", phases=None, precision: str = "f64") -> Problem:
    """2D moire QSE lifted to n=4: V(y)=eps sum_{j<=4} cos(y_j+phi_j), 16 eigenpairs."""
    m, c = cosine_modes(4, eps, phases)
    return Problem("moire2d", moire_P(theta), (K, K), (L, L), m, c, nev=16, block=16,
                   method=method, precision=precision,
                   meta={"eps": eps, "theta": theta})


def config_3d(eps: float = 3.0, K: int = 8, L: int = 8, precision: str = "c64") -> Problem:
    """3D QSE lifted to n=6, P=[I_3, sqrt2 I_3], V=eps sum_j (cos y_j + cos y_{j+3})."""
    P = np.concatenate([np.eye(3), math.sqrt(2.0) * np.eye(3)], axis=1)
    m, c = cosine_modes(6, eps)
    return Problem("qse3d", P, (K, K, K), (L, L, L), m, c, nev=16, block=16,
                   precision=precision, meta={"eps": eps})


def example_41(v0: float = 2.5, K: int = 5, L: int = 60, method: str = "iwfpm",
               shift_round: bool = False) -> Problem:
    """Example 4.1: v = v0[2 - cos 2pi x - cos 2pi alpha x], P = 2pi(1, alpha)."""
    P = 2.0 * math.pi * np.array([[1.0, ALPHA_EX41]])
    m, c = cosine_modes(2, -v0, const=2.0 * v0)
    return Problem("ex41", P, (K,), (L,), m, c, method=method, shift_round=shift_round,
                   meta={"v0": v0})


def example_42(beta: float, theta: float, K: int = 6, L: int = 20, method: str = "iwfpm",
               shift_round: bool = False) -> Problem:
    """Example 4.2: v = 4 - [cos b x1 + 2 cos b x2 + cos(b x1 cos t + b x2 sin t)],
    P = b [[1, 0, cos t], [0, 1, sin t]], V(y) = 4 - (cos y1 + 2 cos y2 + cos y3)."""
    c, s = math.cos(theta), math.sin(theta)
    if abs(theta - math.pi / 4) < 1e-15:
        c = s = math.sqrt(0.5)
    P = beta * np.array([[1.0, 0.0, c], [0.0, 1.0, s]])
    m, co = cosine_modes(3, [-1.0, -2.0, -1.0], const=4.0)
    return Problem("ex42", P, (K, K), (L,), m, co, method=method, shift_round=shift_round,
                   meta={"beta": beta, "theta": theta})


def example_43(beta: float, K: int = 5, L: int = 10, theta: float = 0.2 * math.pi,
               method: str = "iwfpm", shift_round: bool = False) -> Problem:
    """Example 4.3: v = 6 - [cos b x1 + cos b x2 + cos b x3 + cos(b x1 cos t + b x2 sin t)
    + cos(-b x1 sin t + b x2 cos t) + cos(b alpha x3)], t = 0.2 pi, V(y) = 6 - sum_j cos y_j."""
    c, s = math.cos(theta), math.sin(theta)
    P = beta * np.array([[1.0, 0.0, 0.0, c, -s, 0.0],
                         [0.0, 1.0, 0.0, s, c, 0.0],
                         [0.0, 0.0, 1.0, 0.0, 0.0, ALPHA_EX41]])
    m, co = cosine_modes(6, -1.0, const=6.0)
    return Problem("ex43", P, (K, K, K), (L, L, L), m, co, method=method,
                   shift_round=shift_round, meta={"beta": beta, "theta": theta})


def sweep_params(count: int, seed: int):
    """Batched moire sweep: eps ~ U[0.1,10], phases ~ U[0,2pi)^4, cutoff c ~ U[8,20].

    The cutoff maps to K = L = floor(0.65 c + 1/2), so the lifted grids (2K)^4 span
    roughly 10^4 .. 4.6x10^5 points.
    """
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.1, 10.0, size=count)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=(count, 4))
    cut = rng.uniform(8.0, 20.0, size=count)
    KL = np.floor(0.65 * cut + 0.5).astype(np.int64)
    return eps, phases, cut, KL


def sweep_problem(eps: float, phases, KL: int, precision: str = "c64") -> Problem:
    return config_moire(eps=float(eps), K=int(KL), L=int(KL), phases=phases,
                        precision=precision)


def random_block(N: int, nvec: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """Seeded complex-normal block, column-major (N, nvec) layout as a Fortran array."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((nvec, N)) + 1j * rng.standard_normal((nvec, N))
    return np.ascontiguousarray(x.astype(dtype)).T  # (N, nvec), each column contiguous


def physical_grid(d: int, h: float = 0.1, half_width: float | None = None,
                  rows: int | None = None) -> np.ndarray:
    """Uniform grid on [-5a, 5a]^d, a = 10^(3-d), step h (the observation grid of Sec. 4.2:
    10001 points in 1D, 1001^2 in 2D, 101^3 in 3D), as an (M, d) array, last axis fastest.
    `rows` keeps only the first rows of the slowest axis (a bounded sample of the grid)."""
    hw = 5.0 * 10.0 ** (3 - d) if half_width is None else half_width
    cnt = int(round(2 * hw / h)) + 1
    axis = -hw + h * np.arange(cnt)
    axes = [axis[:rows] if (rows is not None and j == 0) else axis for j in range(d)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ascontiguousarray(np.stack([g.ravel() for g in mesh], axis=1))


def grid_descriptor(d: int, rows: int | None = None, h: float = 0.1):
    """(origin, step, count) of the 2D observation grid [-5a, 5a]^2, a = 10^(3-d), step h, as a
    uniform-grid evaluation takes it: the same points, in the same order, as
    physical_grid(d, h, rows=rows)."""
    hw = 5.0 * 10.0 ** (3 - d)
    cnt = int(round(2 * hw / h)) + 1
    return (-hw, -hw), (h, h), (min(cnt, rows or cnt), cnt)


def random_P(d: int, n: int, seed: int) -> np.ndarray:
    """P = [I_d, Q0] with Q0 ~ U(-1.5, 1.5): generic irrational-looking entries."""
    rng = np.random.default_rng(seed)
    return np.concatenate([np.eye(d), rng.uniform(-1.5, 1.5, size=(d, n - d))], axis=1)


def random_modes(n: int, count: int, radius: int, seed: int):
    """A real random potential: count +-m pairs with |m_j| <= radius, plus a real constant."""
    available = ((2 * radius + 1) ** n - 1) // 2
    if count > available:
        raise ValueError(f"only {available} +-m pairs exist with |m_j| <= {radius} in {n}-D")
    rng = np.random.default_rng(seed)
    modes, coef = [[0] * n], [complex(rng.standard_normal())]
    seen = {tuple([0] * n)}
    while len(modes) < 1 + 2 * count:
        m = tuple(int(v) for v in rng.integers(-radius, radius + 1, size=n))
        if m in seen or tuple(-v for v in m) in seen:
            continue
        seen.add(m)
        c = complex(rng.standard_normal(), rng.standard_normal()) * 0.5
        modes.append(list(m))
        coef.append(c)
        modes.append([-v for v in m])
        coef.append(c.conjugate())
    return np.asarray(modes, dtype=np.int64), np.asarray(coef, dtype=np.complex128)


def warmstart_features(eps, phases, width: int = 64) -> np.ndarray:
    """Inputs of the warm-start network for potentials eps * sum_j cos(y_j + phi_j).

    Row per problem: [eps/10, log10(eps), sqrt(eps/10), cos phi_1..4, sin phi_1..4],
    zero-padded to `width` columns. Most of the phase dependence is removed before the
    network by a diagonal unitary on the coefficients (exact for grid-lattice phases); the
    network learns the rest.
    """
    eps = np.atleast_1d(np.asarray(eps, dtype=np.float64))
    phases = np.atleast_2d(np.asarray(phases, dtype=np.float64))
    q = phases.shape[1]
    f = np.zeros((eps.size, width), dtype=np.float32)
    f[:, 0] = eps / 10.0
    f[:, 1] = np.log10(eps)
    f[:, 2] = np.sqrt(eps / 10.0)
    f[:, 3:3 + q] = np.cos(phases)
    f[:, 3 + q:3 + 2 * q] = np.sin(phases)
    return f
