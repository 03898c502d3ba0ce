"""CPU oracle for the IWFPM hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 restatement of what the paper (arXiv 2404.04507) computes:
the irrational window and its index-shift map (Sec. 3.1-3.2), the discrete transform
F = T F* of Algorithm 1 (Sec. 3.3), the discretised Hamiltonian
H~ = Lambda + F V F^{-1} (Sec. 4.1) written as a direct spectral convolution (no FFT),
the diagonal preconditioner (Eq. precond) and reference eigenpairs.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline / reference arm
may import this package. The product path (the CUDA library and its Python binding)
never imports, links or calls anything here, and this package never imports the product.
Inputs come from ``paper_2404_04507_gb300.workloads``, which states problems only.
"""
from .window import Window, WindowTie, build_window, brute_force_window, split_Q
from .operator import (grid_coefficients, apply_stencil, dense_matrix, precond_diag,
                       potential_shift)
from . import transform, eigen

__all__ = ["Window", "WindowTie", "build_window", "brute_force_window", "split_Q",
           "grid_coefficients", "apply_stencil", "dense_matrix", "precond_diag",
           "potential_shift", "transform", "eigen"]
