"""GB300 (sm_103a) implementation of the IWFPM hot path (arXiv 2404.04507).

``Plan`` wraps the C ABI of ``include/iwfpm.h``: it marshals numpy/torch arguments into the
library's calls and nothing more. Device buffers are torch CUDA tensors; the CUDA library
does every step of the computation. Importing ``Plan`` requires the built library.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

__all__ = ["Plan", "gram", "block_update", "batch_solve"]


def _torch():
    import torch
    return torch


def _solve_precision(c, precision):
    """Solver precision names: "f64" (tensor-core contractions), "c64" (complex-float first
    phase), "f64_df" (double-float contractions) or "f64_exact" (FP64 contractions)."""
    table = {"f64": c.IWF_PREC_F64, "c64": c.IWF_PREC_C64, "f64_exact": c.IWF_PREC_F64_EXACT,
             "f64_df": c.IWF_PREC_F64_DF}
    if precision not in table:
        raise ValueError(f"precision must be one of {sorted(table)}")
    return table[precision]


class Plan:
    """A window plan: P (d x n), K (d), L (n-d), method and shift mode (Sec. 3.1-3.2)."""

    def __init__(self, P, K, L, method: str = "iwfpm", shift_round: bool = False,
                 device: int = 0):
        from . import capi
        self._c = capi
        P = np.ascontiguousarray(np.asarray(P, dtype=np.float64))
        d, n = P.shape
        K = np.ascontiguousarray(np.asarray(K, dtype=np.int32).reshape(d))
        L = np.ascontiguousarray(np.asarray(L, dtype=np.int32).reshape(n - d))
        opts = capi.iwf_plan_opts(capi.IWF_METHOD_PM if method == "pm" else capi.IWF_METHOD_IWFPM,
                                  capi.IWF_SHIFT_ROUND if shift_round else capi.IWF_SHIFT_EXACT,
                                  int(device))
        h = C.c_void_p()
        capi.check(capi.iwf_plan_create(C.byref(h), d, n,
                                        P.ctypes.data_as(C.POINTER(C.c_double)),
                                        K.ctypes.data_as(C.POINTER(C.c_int)),
                                        L.ctypes.data_as(C.POINTER(C.c_int)), C.byref(opts)),
                   "iwf_plan_create")
        self.handle = h
        self.d, self.n, self.device = d, n, int(device)
        N = C.c_longlong()
        capi.check(capi.iwf_plan_size(h, C.byref(N)), "iwf_plan_size")
        self.N = int(N.value)
        lens = (C.c_int * n)()
        capi.check(capi.iwf_plan_lens(h, lens), "iwf_plan_lens")
        self.lens = tuple(int(v) for v in lens)

    def close(self):
        if getattr(self, "handle", None):
            self._c.iwf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def window(self) -> np.ndarray:
        k = np.empty((self.N, self.n), dtype=np.int32)
        self._c.check(self._c.iwf_window(self.handle, k.ctypes.data_as(C.POINTER(C.c_int))),
                      "iwf_window")
        return k

    def kinetic(self) -> np.ndarray:
        lam = np.empty(self.N, dtype=np.float64)
        self._c.check(self._c.iwf_kinetic(self.handle, lam.ctypes.data_as(C.POINTER(C.c_double))),
                      "iwf_kinetic")
        return lam

    def set_potential(self, modes, coef):
        modes = np.ascontiguousarray(np.asarray(modes, dtype=np.int32).reshape(-1, self.n))
        coef = np.asarray(coef, dtype=np.complex128).reshape(-1)
        re = np.ascontiguousarray(coef.real)
        im = np.ascontiguousarray(coef.imag)
        self._c.check(self._c.iwf_set_potential(self.handle, int(modes.shape[0]),
                                                modes.ctypes.data_as(C.POINTER(C.c_int)),
                                                re.ctypes.data_as(C.POINTER(C.c_double)),
                                                im.ctypes.data_as(C.POINTER(C.c_double))),
                      "iwf_set_potential")

    def preconditioner(self):
        M = np.empty(self.N, dtype=np.float64)
        sigma = C.c_double()
        self._c.check(self._c.iwf_preconditioner(self.handle,
                                                 M.ctypes.data_as(C.POINTER(C.c_double)),
                                                 C.byref(sigma)), "iwf_preconditioner")
        return M, float(sigma.value)

    @staticmethod
    def _stream(stream):
        if stream is None:
            return C.c_void_p(_torch().cuda.current_stream().cuda_stream)
        if hasattr(stream, "cuda_stream"):          # torch.cuda.Stream
            return C.c_void_p(stream.cuda_stream)
        return C.c_void_p(int(stream))

    def _prec(self, t):
        torch = _torch()
        if t.dtype == torch.complex128:
            return self._c.IWF_PREC_F64
        if t.dtype == torch.complex64:
            return self._c.IWF_PREC_C64
        raise TypeError("vectors must be complex128 or complex64 tensors")

    def _check_block(self, t):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("expected a CUDA tensor")
        nvec = 1 if t.dim() == 1 else t.shape[0]
        if t.numel() != nvec * self.N or not t.is_contiguous():
            raise ValueError("expected a contiguous (nvec, N) block in window order")
        return nvec

    def evaluate(self, coef, x, out=None, stream=None):
        """iwf_evaluate: u(x) = sum_k coef_k exp(i (P k).x) at the rows of x (M, d), for a
        complex128 CUDA vector coef (N,) in window order; returns a complex128 CUDA (M,)."""
        torch = _torch()
        if not (isinstance(coef, torch.Tensor) and coef.is_cuda and coef.dtype == torch.complex128
                and coef.numel() == self.N and coef.is_contiguous()):
            raise TypeError("coef must be a contiguous complex128 CUDA vector of length N")
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64
                and x.dim() == 2 and x.is_contiguous()):
            raise TypeError("x must be a contiguous float64 CUDA tensor of shape (M, d)")
        if x.shape[1] != self.d:
            raise ValueError("x must have d = %d columns" % self.d)
        M = x.shape[0]
        if out is None:
            out = torch.empty(M, dtype=torch.complex128, device=coef.device)
        elif not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.complex128
                  and out.numel() == M and out.is_contiguous()):
            raise TypeError("out must be a contiguous complex128 CUDA vector of length M")
        self._c.check(self._c.iwf_evaluate(self.handle, C.c_void_p(coef.data_ptr()),
                                           C.c_void_p(x.data_ptr()), int(M),
                                           C.c_void_p(out.data_ptr()), self._stream(stream)),
                      "iwf_evaluate")
        return out

    def evaluate_grid(self, coef, origin, step, count, out=None, stream=None):
        """iwf_evaluate_grid: u on the uniform grid origin + (a step_0, b step_1), 0 <= a <
        count[0], 0 <= b < count[1], for d = 2 and a diagonal P_I; returns a complex128 CUDA
        vector of count[0]*count[1] values, the last axis fastest."""
        torch = _torch()
        if not (isinstance(coef, torch.Tensor) and coef.is_cuda and coef.dtype == torch.complex128
                and coef.numel() == self.N and coef.is_contiguous()):
            raise TypeError("coef must be a contiguous complex128 CUDA vector of length N")
        o = (C.c_double * 2)(*[float(v) for v in origin])
        h = (C.c_double * 2)(*[float(v) for v in step])
        n = (C.c_int * 2)(*[int(v) for v in count])
        M = int(count[0]) * int(count[1])
        if out is None:
            out = torch.empty(max(M, 0), dtype=torch.complex128, device=coef.device)
        elif not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.complex128
                  and out.numel() == M and out.is_contiguous()):
            raise TypeError("out must be a contiguous complex128 CUDA vector of count[0]*count[1]")
        self._c.check(self._c.iwf_evaluate_grid(self.handle, C.c_void_p(coef.data_ptr()), o, h, n,
                                                C.c_void_p(out.data_ptr()), self._stream(stream)),
                      "iwf_evaluate_grid")
        return out

    @staticmethod
    def _check_field(u, name):
        torch = _torch()
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dtype == torch.complex128
                and u.dim() == 1 and u.is_contiguous()):
            raise TypeError(name + " must be a contiguous complex128 CUDA vector")

    def normalize_field(self, u, at=None, want_rho=True, stream=None):
        """iwf_field_normalize: u <- u / u[i*] in place, i* = `at` if given, else the first
        point of largest |u|; returns (rho = |u|^2 or None, i* as a CUDA int64 tensor)."""
        torch = _torch()
        self._check_field(u, "u")
        M = u.shape[0]
        rho = torch.empty(M, dtype=torch.float64, device=u.device) if want_rho else None
        idx = torch.empty(1, dtype=torch.int64, device=u.device)
        self._c.check(self._c.iwf_field_normalize(
            self.handle, C.c_void_p(u.data_ptr()), int(M), -1 if at is None else int(at),
            C.c_void_p(rho.data_ptr() if rho is not None else 0), C.c_void_p(idx.data_ptr()),
            self._stream(stream)), "iwf_field_normalize")
        return rho, idx

    def field_distance(self, u, v, stream=None):
        """iwf_field_distance: E_f = max |u - v| as a CUDA float64 tensor of one element."""
        torch = _torch()
        self._check_field(u, "u")
        self._check_field(v, "v")
        if u.shape != v.shape:
            raise ValueError("u and v must have the same length")
        out = torch.empty(1, dtype=torch.float64, device=u.device)
        self._c.check(self._c.iwf_field_distance(
            self.handle, C.c_void_p(u.data_ptr()), C.c_void_p(v.data_ptr()), int(u.shape[0]),
            C.c_void_p(out.data_ptr()), self._stream(stream)), "iwf_field_distance")
        return out

    def apply_stencil(self, psi, out=None, stream=None):
        """iwf_apply_stencil: H~ psi by direct convolution with the folded modes (few-mode
        potentials); same layout and result as apply()."""
        nvec = self._check_block(psi)
        if out is None:
            out = _torch().empty_like(psi)
        self._check_block(out)
        if out.dtype != psi.dtype:
            raise TypeError("psi and out must share a dtype")
        self._c.check(self._c.iwf_apply_stencil(self.handle, self._prec(psi),
                                                C.c_void_p(psi.data_ptr()),
                                                C.c_void_p(out.data_ptr()), int(nvec),
                                                self._stream(stream)), "iwf_apply_stencil")
        return out

    def apply_host(self, psi, out=None, stream=None):
        """iwf_apply_host: H~ psi for a contiguous (nvec, N) or (N,) complex CPU tensor
        (pinned memory gives the full copy bandwidth); returns when `out` is complete."""
        torch = _torch()
        if not isinstance(psi, torch.Tensor) or psi.is_cuda:
            raise TypeError("expected a CPU tensor")
        nvec = 1 if psi.dim() == 1 else psi.shape[0]
        if psi.numel() != nvec * self.N or not psi.is_contiguous():
            raise ValueError("expected a contiguous (nvec, N) block in window order")
        if out is None:
            out = torch.empty_like(psi, pin_memory=psi.is_pinned())
        if out.is_cuda or out.dtype != psi.dtype or out.shape != psi.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous CPU tensor like psi")
        self._c.check(self._c.iwf_apply_host(self.handle, self._prec(psi), C.c_void_p(psi.data_ptr()),
                                             C.c_void_p(out.data_ptr()), int(nvec),
                                             self._stream(stream)), "iwf_apply_host")
        return out

    def apply(self, psi, out=None, stream=None):
        """H~ psi for a contiguous (nvec, N) or (N,) complex CUDA tensor (window order)."""
        nvec = self._check_block(psi)
        if out is None:
            out = _torch().empty_like(psi)
        self._check_block(out)
        if out.dtype != psi.dtype:
            raise TypeError("psi and out must share a dtype")
        self._c.check(self._c.iwf_apply(self.handle, self._prec(psi), C.c_void_p(psi.data_ptr()),
                                        C.c_void_p(out.data_ptr()), int(nvec),
                                        self._stream(stream)), "iwf_apply")
        return out

    def autotune(self, precision="f64", nvec=16, stream=None):
        """iwf_plan_autotune: returns (ms per apply, (threads, tile_kb, chunk_mb))."""
        ms = C.c_double()
        best = (C.c_int * 3)()
        prec = self._c.IWF_PREC_F64 if precision == "f64" else self._c.IWF_PREC_C64
        self._c.check(self._c.iwf_plan_autotune(self.handle, prec, int(nvec), C.byref(ms), best,
                                                self._stream(stream)), "iwf_plan_autotune")
        return float(ms.value), tuple(int(v) for v in best)

    def set_schedule(self, precision, threads, tile_kb, chunk_mb):
        prec = self._c.IWF_PREC_F64 if precision == "f64" else self._c.IWF_PREC_C64
        self._c.check(self._c.iwf_plan_set_schedule(self.handle, prec, int(threads),
                                                    int(tile_kb), int(chunk_mb)),
                      "iwf_plan_set_schedule")

    _PATHS = {"auto": 0, "tiled": 1, "pencil": 2}

    def set_path(self, precision, path):
        """iwf_plan_set_path: path is "auto", "tiled" or "pencil"."""
        prec = self._c.IWF_PREC_F64 if precision == "f64" else self._c.IWF_PREC_C64
        self._c.check(self._c.iwf_plan_set_path(self.handle, prec, self._PATHS[path]),
                      "iwf_plan_set_path")

    def schedule(self, precision):
        """iwf_plan_get_schedule: dict with threads, tile_kb, chunk_mb and path."""
        prec = self._c.IWF_PREC_F64 if precision == "f64" else self._c.IWF_PREC_C64
        out = (C.c_int * 4)()
        self._c.check(self._c.iwf_plan_get_schedule(self.handle, prec, out),
                      "iwf_plan_get_schedule")
        names = {1: "tiled", 2: "pencil"}
        return {"threads": out[0], "tile_kb": out[1], "chunk_mb": out[2],
                "path": names[out[3]]}

    def set_arith(self, arith):
        """iwf_plan_set_arith: "f64" or "df" (double-float DFTs of FP64 applies, pencil path)."""
        code = {"f64": 0, "df": 1}[arith]
        self._c.check(self._c.iwf_plan_set_arith(self.handle, code), "iwf_plan_set_arith")

    def coef_extent(self, coef, threshold, stream=None):
        """iwf_coef_extent: per axis, the smallest half-width (K'_j, then L'_j) of a window
        with this plan's centring that holds every coefficient with |c_k| >= threshold
        (coef: a complex128 CUDA tensor of N values in window order)."""
        torch = _torch()
        if not isinstance(coef, torch.Tensor) or not coef.is_cuda or coef.dtype != torch.complex128:
            raise TypeError("coef must be a complex128 CUDA tensor")
        c = coef.contiguous()
        if c.numel() != self.N:
            raise ValueError("coef must hold N values")
        need = (C.c_int * self.n)()
        self._c.check(self._c.iwf_coef_extent(self.handle, C.c_void_p(c.data_ptr()),
                                              float(threshold), need, self._stream(stream)),
                      "iwf_coef_extent")
        return np.array(list(need), dtype=np.int64)

    def trim(self):
        """iwf_plan_trim: free the eigensolver workspace kept on the plan between solves."""
        self._c.iwf_plan_trim(self.handle)

    def check(self, stream=None):
        """iwf_plan_check: raises IwfError (IWF_ERR_TIMEOUT) if an apply on this plan gave up
        waiting since the last check; synchronises the stream."""
        self._c.check(self._c.iwf_plan_check(self.handle, self._stream(stream)), "iwf_plan_check")

    def set_wait_limit(self, rounds):
        """iwf_plan_set_wait_limit: try_wait rounds of each main wait of the pipelined passes
        (negative: the default)."""
        self._c.check(self._c.iwf_plan_set_wait_limit(self.handle, int(rounds)),
                      "iwf_plan_set_wait_limit")

    def apply_profile(self, psi, out, stream=None):
        """iwf_apply_profile: same result as apply(); returns (pass_ms[3], launches[3])."""
        nvec = self._check_block(psi)
        self._check_block(out)
        ms = (C.c_double * 3)()
        nl = (C.c_int * 3)()
        self._c.check(self._c.iwf_apply_profile(self.handle, self._prec(psi),
                                                C.c_void_p(psi.data_ptr()),
                                                C.c_void_p(out.data_ptr()), int(nvec),
                                                self._stream(stream), ms, nl),
                      "iwf_apply_profile")
        return [float(v) for v in ms], [int(v) for v in nl]


    def eigensolve(self, nev, block=0, tol=1e-10, maxit=0, precision="f64", c64_tol=0.0,
                   seed=1, X0=None, stream=None, raise_noconv=True):
        """Lowest nev eigenpairs (iwf_eigensolve). Returns (evals, evecs (nev, N), resid, info)."""
        torch = _torch()
        c = self._c
        opts = c.iwf_solve_opts(int(nev), int(block), int(maxit), float(tol),
                                _solve_precision(c, precision),
                                float(c64_tol), int(seed))
        evals = np.zeros(nev)
        resid = np.zeros(nev)
        evecs = torch.empty((nev, self.N), dtype=torch.complex128, device=f"cuda:{self.device}")
        info = c.iwf_solve_info()
        x0 = C.c_void_p(X0.data_ptr()) if X0 is not None else None
        st = c.iwf_eigensolve(self.handle, C.byref(opts), x0,
                              evals.ctypes.data_as(C.POINTER(C.c_double)),
                              C.c_void_p(evecs.data_ptr()),
                              resid.ctypes.data_as(C.POINTER(C.c_double)), C.byref(info),
                              self._stream(stream))
        if st != 0 and not (st == -7 and not raise_noconv):
            c.check(st, "iwf_eigensolve")
        out = {f: getattr(info, f) for f, _ in c.iwf_solve_info._fields_}
        return evals, evecs, resid, out


    def batch_eigensolve(self, potentials, nev, block=0, tol=1e-10, maxit=0, precision="f64",
                         c64_tol=0.0, seed=1, want_vectors=False, stream=None,
                         raise_noconv=True, X0=None):
        """iwf_batch_eigensolve over [(modes, coef), ...] sharing this plan's geometry.

        Returns (evals (nprob, nev), evecs (nprob, nev, N) or None, resid, iters, info)."""
        torch = _torch()
        c = self._c
        nprob = len(potentials)
        nm = np.array([len(np.asarray(cf).reshape(-1)) for _, cf in potentials], dtype=np.int32)
        modes = np.ascontiguousarray(np.concatenate(
            [np.asarray(mm, dtype=np.int32).reshape(-1, self.n) for mm, _ in potentials]))
        coef = np.concatenate([np.asarray(cf, dtype=np.complex128).reshape(-1)
                               for _, cf in potentials])
        re, im = np.ascontiguousarray(coef.real), np.ascontiguousarray(coef.imag)
        opts = c.iwf_solve_opts(int(nev), int(block), int(maxit), float(tol),
                                _solve_precision(c, precision),
                                float(c64_tol), int(seed))
        evals = np.zeros((nprob, nev))
        resid = np.zeros((nprob, nev))
        iters = np.zeros(nprob, dtype=np.int32)
        evecs = None
        if want_vectors:
            evecs = torch.empty((nprob, nev, self.N), dtype=torch.complex128,
                                device=f"cuda:{self.device}")
        info = c.iwf_solve_info()
        st = c.iwf_batch_eigensolve(
            self.handle, nprob, nm.ctypes.data_as(C.POINTER(C.c_int)),
            modes.ctypes.data_as(C.POINTER(C.c_int)), re.ctypes.data_as(C.POINTER(C.c_double)),
            im.ctypes.data_as(C.POINTER(C.c_double)), C.byref(opts),
            C.c_void_p(X0.data_ptr()) if X0 is not None else None,
            evals.ctypes.data_as(C.POINTER(C.c_double)),
            C.c_void_p(evecs.data_ptr()) if evecs is not None else None,
            resid.ctypes.data_as(C.POINTER(C.c_double)), iters.ctypes.data_as(C.POINTER(C.c_int)),
            C.byref(info), self._stream(stream))
        if st != 0 and not (st == -7 and not raise_noconv):
            c.check(st, "iwf_batch_eigensolve")
        out = {f: getattr(info, f) for f, _ in c.iwf_solve_info._fields_}
        return evals, evecs, resid, iters, out


def batch_solve(plans, nev, block=0, tol=1e-10, maxit=0, precision="f64", c64_tol=0.0,
                seed=1, X0=None, want_vectors=False, stream=None, raise_noconv=True):
    """iwf_batch_solve over independent plans (each with its own window and potential).

    Returns (evals (nplans, nev), evecs list or None, resid, iters, info)."""
    from . import capi
    torch = _torch()
    n = len(plans)
    handles = (C.c_void_p * n)(*[p.handle.value for p in plans])
    opts = capi.iwf_solve_opts(int(nev), int(block), int(maxit), float(tol),
                               _solve_precision(capi, precision), float(c64_tol), int(seed))
    evals = np.zeros((n, nev))
    resid = np.zeros((n, nev))
    iters = np.zeros(n, dtype=np.int32)
    x0 = None
    if X0 is not None:
        x0 = (C.c_void_p * n)(*[(x.data_ptr() if x is not None else None) for x in X0])
    vecs = None
    vptr = None
    if want_vectors:
        vecs = [torch.empty((nev, p.N), dtype=torch.complex128, device=f"cuda:{p.device}")
                for p in plans]
        vptr = (C.c_void_p * n)(*[v.data_ptr() for v in vecs])
    info = capi.iwf_solve_info()
    st = capi.iwf_batch_solve(n, handles, C.byref(opts), x0,
                              evals.ctypes.data_as(C.POINTER(C.c_double)), vptr,
                              resid.ctypes.data_as(C.POINTER(C.c_double)),
                              iters.ctypes.data_as(C.POINTER(C.c_int)), C.byref(info),
                              Plan._stream(stream))
    if st != 0 and not (st == -7 and not raise_noconv):
        capi.check(st, "iwf_batch_solve")
    out = {f: getattr(info, f) for f, _ in capi.iwf_solve_info._fields_}
    return evals, vecs, resid, iters, out


_ENGINES = {"tensor": 0, "df": 1, "f64": 2}


def _contract_args(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def gram(A, B, engine="tensor", stream=None):
    """iwf_gram: G = A^H B for blocks given as (columns, nrows) complex128 CUDA tensors (each
    row of the tensor is one column of the matrix). Returns G (ma, mb) on the device."""
    from . import capi
    torch = _torch()
    _contract_args(A, "A"); _contract_args(B, "B")
    ma, nrows = A.shape
    mb = B.shape[0]
    if B.shape[1] != nrows:
        raise ValueError("A and B need the same number of rows")
    G = torch.empty((ma, mb), dtype=torch.complex128, device=A.device)
    capi.check(capi.iwf_gram(_ENGINES[engine], int(nrows), C.c_void_p(A.data_ptr()), int(ma),
                             C.c_void_p(B.data_ptr()), int(mb), C.c_void_p(G.data_ptr()),
                             A.device.index or 0, Plan._stream(stream)), "iwf_gram")
    return G


def block_update(S, Cm, Y=None, subtract=False, engine="tensor", stream=None):
    """iwf_block_update: Y = S C (or Y -= S C) with S (m, nrows) and Y (q, nrows) given as
    column blocks and C an (m, q) complex128 CUDA tensor (row-major). Returns Y."""
    from . import capi
    torch = _torch()
    _contract_args(S, "S"); _contract_args(Cm, "C")
    m, nrows = S.shape
    q = Cm.shape[1]
    if Cm.shape[0] != m:
        raise ValueError("C must have one row per column of S")
    if Y is None:
        if subtract:
            raise ValueError("subtract needs Y")
        Y = torch.empty((q, nrows), dtype=torch.complex128, device=S.device)
    _contract_args(Y, "Y")
    capi.check(capi.iwf_block_update(_ENGINES[engine], int(nrows), C.c_void_p(S.data_ptr()),
                                     int(m), C.c_void_p(Cm.data_ptr()), int(q),
                                     C.c_void_p(Y.data_ptr()), int(bool(subtract)),
                                     S.device.index or 0, Plan._stream(stream)),
               "iwf_block_update")
    return Y


def kernel_launches() -> int:
    """Kernels launched by the CUDA library so far in this process."""
    from . import capi
    return int(capi.iwf_kernel_launches())
