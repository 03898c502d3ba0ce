"""ctypes wrapper of ``capply.c``: the oracle's direct-convolution H~ psi in plain C with
OpenMP over the host's cores (oracle; test infrastructure only).

Same operator and mode order as ``operator.apply_stencil`` (Sec. 4.1, Sec. 3.3, App. C);
``build()`` compiles the shared library with gcc, ``apply()`` calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .window import Window

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "capply.c")
LIB = os.path.join(HERE, "liboracle_apply.so")


def build() -> str:
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC],
                       check=True, capture_output=True, text=True)
    return LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.oracle_apply.restype = C.c_int
        _lib.oracle_apply.argtypes = [C.c_longlong, C.c_int] + [C.c_void_p] * 3 + \
            [C.c_int] + [C.c_void_p] * 3 + [C.c_int, C.c_void_p, C.c_void_p]
    return _lib


def apply(win: Window, Vg: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """H~ psi for psi (N,) or (N, nvec) complex in window order."""
    lib = _load()
    X = np.asarray(psi, dtype=np.complex128)
    vec = X.ndim == 1
    X = np.asfortranarray(X[:, None] if vec else X)
    shifts = np.argwhere(Vg != 0).astype(np.int32)
    coef = Vg[tuple(shifts.T)] if len(shifts) else np.zeros(0, np.complex128)
    lens = np.ascontiguousarray(np.asarray(win.lens, dtype=np.int32))
    kstar = np.ascontiguousarray(win.kstar.astype(np.int32))
    lam = np.ascontiguousarray(win.lam, dtype=np.float64)
    sh = np.ascontiguousarray(shifts)
    vre = np.ascontiguousarray(coef.real)
    vim = np.ascontiguousarray(coef.imag)
    out = np.empty_like(X, order="F")
    st = lib.oracle_apply(win.N, len(win.lens), lens.ctypes.data, kstar.ctypes.data,
                          lam.ctypes.data, len(shifts), sh.ctypes.data, vre.ctypes.data,
                          vim.ctypes.data, X.shape[1], X.ctypes.data, out.ctypes.data)
    if st != 0:
        raise MemoryError("oracle_apply: allocation failed")
    return out[:, 0] if vec else out
