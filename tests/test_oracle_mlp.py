"""Pins of the warm-start oracle: backpropagation vs central finite differences, and the
subspace loss vs its definition (zero for a rotated copy of the reference block)."""
import numpy as np

from oracle import mlp


def _setup(seed=0):
    rng = np.random.default_rng(seed)
    dims = [5, 7, 6, 2 * 3 * 4]      # nvec = 3, ncore = 4
    n = sum(a * c + c for a, c in zip(dims[:-1], dims[1:]))
    flat = rng.standard_normal(n) * 0.4
    feats = rng.standard_normal((4, 5))
    X = rng.standard_normal((4, dims[-1]))
    return dims, flat, feats, X


def test_backprop_matches_finite_differences():
    dims, flat, feats, X = _setup()
    loss, g = mlp.loss_and_grad(flat, dims, feats, X, 3, 4)
    h = 1e-6
    for i in np.random.default_rng(1).choice(flat.size, 25, replace=False):
        e = np.zeros_like(flat); e[i] = h
        lp, _ = mlp.loss_and_grad(flat + e, dims, feats, X, 3, 4)
        lm, _ = mlp.loss_and_grad(flat - e, dims, feats, X, 3, 4)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_subspace_loss_is_gauge_invariant():
    rng = np.random.default_rng(3)
    ncore, nvec = 10, 3
    q, _ = np.linalg.qr(rng.standard_normal((ncore, nvec)) + 1j * rng.standard_normal((ncore, nvec)))
    u, _ = np.linalg.qr(rng.standard_normal((nvec, nvec)) + 1j * rng.standard_normal((nvec, nvec)))
    def flat(m):
        f = np.zeros(2 * ncore * nvec)
        c = m.T.reshape(-1)
        f[0::2], f[1::2] = c.real, c.imag
        return f[None, :]
    loss, _ = mlp.subspace_loss(flat(q @ u), flat(q), nvec, ncore)
    assert abs(loss) < 1e-12
    loss2, _ = mlp.subspace_loss(flat(np.zeros_like(q)), flat(q), nvec, ncore)
    assert abs(loss2 - 1.0) < 1e-12          # |X X^H|^2 / nvec = nvec / nvec


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159265], np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0                                 # a tie goes to even
    assert r[2] == 1.0                                                # below half an ulp
    assert r[3] == 1.0 + 2 ** -7
    assert abs(r[4] + 3.140625) < 1e-12
