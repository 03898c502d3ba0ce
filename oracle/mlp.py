"""Oracle for the learned warm start (test infrastructure only).

A plain numpy MLP -- dense layers with GELU (0.5 z (1 + erf(z / sqrt 2))) between them and a
linear output -- and the gauge-invariant subspace loss used to train it:
    L(Y) = |X X^H - Y Y^H|_F^2 = |X^H X|^2 - 2 |X^H Y|^2 + |Y^H Y|^2   (per sample),
where X (ncore x nvec) are the reference eigenvectors on the window core and Y the
prediction, both read from the flat output vector as o = (v * ncore + i) * 2 + {re, im}.
The loss does not depend on the phase of each eigenvector nor on rotations inside a
degenerate eigenspace, which a plain squared error would penalise. The mean over the batch
is divided by nvec.
Rounding: ``bf16=True`` rounds weights and every layer input to bfloat16 (round to nearest
even on the float32 bit pattern) at the same points as a BF16 tensor-core implementation,
with every product accumulated in float64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def unpack_params(flat, dims):
    """Flat parameters -> [(W (out x in), b (out))] for layer sizes dims[0] -> ... -> dims[-1]."""
    out, off = [], 0
    for a, c in zip(dims[:-1], dims[1:]):
        W = flat[off:off + a * c].reshape(c, a)
        off += a * c
        b = flat[off:off + c]
        off += c
        out.append((W, b))
    assert off == flat.size
    return out


def forward(flat, dims, feats, bf16=False):
    q = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack_params(np.asarray(flat, dtype=np.float64), dims)
    h = q(feats)
    cache = []
    for li, (W, b) in enumerate(layers):
        z = h @ q(W).T + b
        cache.append((h, z))
        h = q(gelu(z)) if li + 1 < len(layers) else z
    return h, cache


def subspace_loss(Y, X, nvec, ncore):
    """Mean over samples of |XX^H - YY^H|_F^2 / nvec and dL/dY (same flat layout)."""
    B = Y.shape[0]
    Yc = (Y[:, 0::2] + 1j * Y[:, 1::2]).reshape(B, nvec, ncore).transpose(0, 2, 1)
    Xc = (X[:, 0::2] + 1j * X[:, 1::2]).reshape(B, nvec, ncore).transpose(0, 2, 1)
    loss, grad = 0.0, np.zeros_like(Y, dtype=np.float64)
    for s in range(B):
        x, y = Xc[s], Yc[s]
        gxx, gxy, gyy = x.conj().T @ x, x.conj().T @ y, y.conj().T @ y
        loss += (np.sum(np.abs(gxx) ** 2) - 2 * np.sum(np.abs(gxy) ** 2)
                 + np.sum(np.abs(gyy) ** 2)).real
        g = (-4.0 * x @ gxy + 4.0 * y @ gyy).T.reshape(-1)   # d/d(Re y) + i d/d(Im y)
        grad[s, 0::2], grad[s, 1::2] = g.real, g.imag
    scale = 1.0 / (B * nvec)
    return loss * scale, grad * scale


def loss_and_grad(flat, dims, feats, X, nvec, ncore, bf16=False):
    """Loss and its gradient with respect to the flat parameters (backpropagation)."""
    q = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    layers = unpack_params(np.asarray(flat, dtype=np.float64), dims)
    Y, cache = forward(flat, dims, feats, bf16)
    loss, dY = subspace_loss(Y, X, nvec, ncore)
    grads = []
    dz = dY
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h, z = cache[li]
        grads.append((dz.T @ h, dz.sum(axis=0)))
        if li:
            dh = dz @ q(W)
            dz = dh * gelu_grad(cache[li - 1][1])
    grads.reverse()
    flat_g = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, flat_g
