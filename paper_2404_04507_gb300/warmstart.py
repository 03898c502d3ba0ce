"""Learned warm start (binding of the iwf_ws_* entry points; marshalling only).

A network trained on the eigenvectors of small "core" windows predicts the start block of
a solve on a larger window: predict on the core, embed by true index (zero elsewhere),
hand to the batched eigensolver as X0 (which orthonormalises it).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import capi


def _torch():
    import torch
    return torch


class WarmStart:
    def __init__(self, dims, seed: int = 1, device: int = 0):
        self.dims = [int(v) for v in dims]
        d = np.ascontiguousarray(np.asarray(self.dims, dtype=np.int32))
        h = C.c_void_p()
        capi.check(capi.iwf_ws_create(C.byref(h), len(dims) - 1,
                                      d.ctypes.data_as(C.POINTER(C.c_int)), int(seed),
                                      int(device)), "iwf_ws_create")
        self.handle, self.device = h, int(device)
        n = C.c_longlong()
        capi.check(capi.iwf_ws_num_params(h, C.byref(n)), "iwf_ws_num_params")
        self.nparams = int(n.value)

    def close(self):
        if getattr(self, "handle", None):
            capi.iwf_ws_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparams, dtype=np.float32)
        capi.check(capi.iwf_ws_get_params(self.handle, out.ctypes.data_as(C.POINTER(C.c_float))),
                   "iwf_ws_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(np.asarray(flat, dtype=np.float32))
        capi.check(capi.iwf_ws_set_params(self.handle, flat.ctypes.data_as(C.POINTER(C.c_float))),
                   "iwf_ws_set_params")

    def _dev(self, a):
        torch = _torch()
        if isinstance(a, torch.Tensor):
            return a.to(device=f"cuda:{self.device}", dtype=torch.float32).contiguous()
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(f"cuda:{self.device}")

    def predict(self, feats):
        torch = _torch()
        f = self._dev(feats)
        out = torch.empty((f.shape[0], self.dims[-1]), dtype=torch.float32, device=f.device)
        capi.check(capi.iwf_ws_predict(self.handle, int(f.shape[0]), C.c_void_p(f.data_ptr()),
                                       C.c_void_p(out.data_ptr()),
                                       C.c_void_p(torch.cuda.current_stream().cuda_stream)),
                   "iwf_ws_predict")
        return out

    def loss_grad(self, feats, targets, nvec, ncore):
        f, t = self._dev(feats), self._dev(targets)
        loss = C.c_float()
        g = np.empty(self.nparams, dtype=np.float32)
        capi.check(capi.iwf_ws_loss_grad(self.handle, int(f.shape[0]), C.c_void_p(f.data_ptr()),
                                         C.c_void_p(t.data_ptr()), int(nvec), int(ncore),
                                         C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_float)),
                                         None), "iwf_ws_loss_grad")
        return float(loss.value), g

    def train(self, feats, targets, nvec, ncore, epochs, batch=64, lr=1e-3, wd=0.0, seed=0):
        torch = _torch()
        f, t = self._dev(feats), self._dev(targets)
        hist = np.zeros(max(epochs, 1), dtype=np.float32)
        capi.check(capi.iwf_ws_train(self.handle, int(f.shape[0]), C.c_void_p(f.data_ptr()),
                                     C.c_void_p(t.data_ptr()), int(nvec), int(ncore), int(epochs),
                                     int(batch), float(lr), float(wd), int(seed),
                                     hist.ctypes.data_as(C.POINTER(C.c_float)),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream)),
                   "iwf_ws_train")
        return hist[:epochs]


def vectors_to_targets(evecs, nvec: int):
    """(nprob, nvec, N) complex eigenvectors -> (nprob, 2*nvec*N) float32 target rows."""
    torch = _torch()
    ev = evecs[:, :nvec, :]
    return torch.view_as_real(ev.contiguous()).reshape(ev.shape[0], -1).to(torch.float32)


def targets_to_vectors(rows, nvec: int, ncore: int):
    """Inverse of vectors_to_targets, complex128 (nprob, nvec, ncore)."""
    torch = _torch()
    r = rows.to(torch.float64).reshape(rows.shape[0], nvec, ncore, 2).contiguous()
    return torch.view_as_complex(r)


def embed(core_plan, big_plan, vecs):
    """(nprob, nvec, core N) complex128 -> (nprob, nvec, big N) by true index."""
    torch = _torch()
    vecs = vecs.to(torch.complex128).contiguous()
    nprob, nvec = int(vecs.shape[0]), int(vecs.shape[1])
    out = torch.empty((nprob, nvec, big_plan.N), dtype=torch.complex128, device=vecs.device)
    capi.check(capi.iwf_ws_embed(core_plan.handle, big_plan.handle, nprob, nvec,
                                 C.c_void_p(vecs.data_ptr()), C.c_void_p(out.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "iwf_ws_embed")
    return out


def phase(plan, vecs, phases, sign: int):
    """In place: vecs[p][v][k] *= exp(i sign k.phi_p) (k the true window index)."""
    torch = _torch()
    assert vecs.dtype == torch.complex128 and vecs.is_contiguous()
    ph = np.ascontiguousarray(np.asarray(phases, dtype=np.float64).reshape(vecs.shape[0], plan.n))
    capi.check(capi.iwf_ws_phase(plan.handle, int(vecs.shape[0]), int(vecs.shape[1]),
                                 ph.ctypes.data_as(C.POINTER(C.c_double)), int(sign),
                                 C.c_void_p(vecs.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream)),
               "iwf_ws_phase")
    return vecs
