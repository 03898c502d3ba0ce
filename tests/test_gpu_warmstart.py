"""Learned warm start: GPU forward/backward against the numpy oracle MLP, training on
eigenvectors the plain solver produces, embedding, and the gain over a cold start.

Gradient tolerance: the oracle rounds weights and layer inputs to bfloat16 at the same
points as the tensor-core GEMMs and accumulates in float64; the GPU also rounds dz to
bfloat16 before the backward GEMMs (unit roundoff 2^-9 per layer) and accumulates in
float32, so the gradients agree to 2e-2 in norm and the loss to 1e-3.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp
from paper_2404_04507_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import paper_2404_04507_gb300 as iwf
    from paper_2404_04507_gb300 import warmstart as ws
    assert torch.cuda.is_available()
    return iwf, ws


def test_gradients_match_oracle(mods):
    _, ws = mods
    dims, nvec, ncore, B = [64, 128, 64, 128], 2, 32, 64
    net = ws.WarmStart(dims, seed=3)
    rng = np.random.default_rng(0)
    flat = mlp.bf16_round(net.get_params()).astype(np.float32)      # bf16-exact weights
    flat += np.where(np.arange(flat.size) % 7 == 0, 0.01, 0.0).astype(np.float32)  # nonzero b
    flat = mlp.bf16_round(flat).astype(np.float32)
    net.set_params(flat)
    feats = mlp.bf16_round(rng.standard_normal((B, dims[0]))).astype(np.float32)
    X = rng.standard_normal((B, dims[-1])).astype(np.float32) * 0.2
    loss, g = net.loss_grad(feats, X, nvec, ncore)
    lref, gref = mlp.loss_and_grad(flat.astype(np.float64), dims, feats.astype(np.float64),
                                   X.astype(np.float64), nvec, ncore, bf16=True)
    assert abs(loss - lref) <= 1e-3 * abs(lref)
    assert np.linalg.norm(g - gref) <= 2e-2 * np.linalg.norm(gref)
    # forward alone
    y = net.predict(feats).cpu().numpy()
    yref, _ = mlp.forward(flat.astype(np.float64), dims, feats.astype(np.float64), bf16=True)
    assert np.max(np.abs(y - yref)) <= 1e-3 * np.max(np.abs(yref))


def test_gradients_match_oracle_long_k_split(mods):
    # the output layer's input gradient contracts over 4096 outputs with only two 128-column
    # tiles: the tensor-core GEMM splits K across CTAs and sums the partial tiles
    _, ws = mods
    dims, nvec, ncore, B = [64, 256, 4096], 2, 1024, 64
    net = ws.WarmStart(dims, seed=5)
    rng = np.random.default_rng(1)
    flat = mlp.bf16_round(net.get_params()).astype(np.float32)
    net.set_params(flat)
    feats = mlp.bf16_round(rng.standard_normal((B, dims[0]))).astype(np.float32)
    X = rng.standard_normal((B, dims[-1])).astype(np.float32) * 0.05
    loss, g = net.loss_grad(feats, X, nvec, ncore)
    lref, gref = mlp.loss_and_grad(flat.astype(np.float64), dims, feats.astype(np.float64),
                                   X.astype(np.float64), nvec, ncore, bf16=True)
    assert abs(loss - lref) <= 1e-3 * abs(lref)
    assert np.linalg.norm(g - gref) <= 2e-2 * np.linalg.norm(gref)
    # the first layer's weights get their gradient through the split-K product
    n0 = dims[0] * dims[1]
    assert np.linalg.norm(g[:n0] - gref[:n0]) <= 2e-2 * np.linalg.norm(gref[:n0])


def _core_dataset(iwf, ws, n, seed, K, nev, block):
    # eigenvectors of the sweep's problems on the core window, with the phases removed by
    # the exact diagonal unitary (targets of the phase-free network)
    eps, phases, _, _ = W.sweep_params(n, seed)
    pb = W.config_moire(eps=1.0, K=K, L=K)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    pots = [W.cosine_modes(4, e, ph) for e, ph in zip(eps, phases)]
    ev, X, res, iters, info = plan.batch_eigensolve(pots, nev, block=block, tol=1e-8,
                                                    want_vectors=True)
    assert info["converged"] == 1
    ws.phase(plan, X, phases, -1)
    return plan, eps, phases, W.warmstart_features(eps, phases), ws.vectors_to_targets(X, nev)


def test_phase_is_the_exact_symmetry_for_grid_lattice_phases(mods):
    # for phi_j in (pi/K) Z the wrap-around of the cyclic grid is consistent, so the phase-
    # shifted phi = 0 eigenvectors are exact eigenvectors of H_phi with the same eigenvalues
    iwf, ws = mods
    K = 6
    pb0 = W.config_moire(eps=2.0, K=K, L=K)
    phases = np.array([1.0, -2.0, 3.0, 5.0]) * math.pi / K
    pb1 = W.config_moire(eps=2.0, K=6, L=6, phases=phases)
    p0 = iwf.Plan(pb0.P, pb0.K, pb0.L); p0.set_potential(pb0.modes, pb0.coef)
    p1 = iwf.Plan(pb1.P, pb1.K, pb1.L); p1.set_potential(pb1.modes, pb1.coef)
    ev0, X0, _, _ = p0.eigensolve(4, block=8)
    X = X0.clone().reshape(1, 4, p0.N)
    ws.phase(p0, X, phases[None, :], +1)
    HX = p1.apply(X[0])
    r = (HX - X[0] * torch.from_numpy(ev0).cuda()[:, None]).norm(dim=1).cpu().numpy()
    assert np.max(r) < 1e-9
    ws.phase(p0, X, phases[None, :], -1)
    assert (X[0] - X0).abs().max().item() < 1e-13


def test_embed_places_by_true_index(mods):
    iwf, ws = mods
    pb2, pb3 = W.config_moire(K=2, L=2), W.config_moire(K=3, L=3)
    core, big = iwf.Plan(pb2.P, pb2.K, pb2.L), iwf.Plan(pb3.P, pb3.K, pb3.L)
    v = torch.randn((2, 3, core.N), dtype=torch.complex128, device="cuda")
    out = ws.embed(core, big, v).cpu().numpy()
    kc, kb = core.window(), big.window()
    pos = {tuple(k): i for i, k in enumerate(kb)}
    idx = np.array([pos[tuple(k)] for k in kc])
    vv = v.cpu().numpy()
    assert np.array_equal(out[:, :, idx], vv)
    mask = np.ones(big.N, bool); mask[idx] = False
    assert np.all(out[:, :, mask] == 0)


def test_training_lowers_loss_and_warm_started_solves_agree(mods):
    # checks that training lowers the loss and that a warm start reaches the cold start's
    # eigenvalues; it does not claim an iteration saving (none is shown at this scale)
    iwf, ws = mods
    nev, K = 4, 2
    plan, _, _, feats, targets = _core_dataset(iwf, ws, 256, 5, K, nev, 8)
    ncore = plan.N
    net = ws.WarmStart([64, 256, 256, 2 * nev * ncore], seed=1)
    hist = net.train(feats, targets, nev, ncore, epochs=150, batch=64, lr=2e-3)
    assert hist[-1] < 0.3 * hist[0], hist[[0, -1]]
    # held-out problems on the larger K = 3 window: warm vs cold iterations
    eps, phases, _, _ = W.sweep_params(64, 6)
    pots = [W.cosine_modes(4, e, ph) for e, ph in zip(eps, phases)]
    pb3 = W.config_moire(K=3, L=3)
    big = iwf.Plan(pb3.P, pb3.K, pb3.L)
    pred = ws.targets_to_vectors(net.predict(W.warmstart_features(eps, phases)), nev, ncore)
    X0 = torch.zeros((64, 8, big.N), dtype=torch.complex128, device="cuda")
    X0[:, :nev] = ws.phase(big, ws.embed(plan, big, pred), phases, +1)
    X0[:, nev:] = torch.randn((64, 8 - nev, big.N), dtype=torch.complex128, device="cuda") * 1e-3
    evw, _, resw, itw, infow = big.batch_eigensolve(pots, nev, block=8, X0=X0)
    evc, _, resc, itc, infoc = big.batch_eigensolve(pots, nev, block=8)
    assert infow["converged"] == 1 and infoc["converged"] == 1
    assert np.allclose(evw, evc, rtol=1e-9, atol=1e-9)
    print(f"warm-start mean iterations {itw.mean():.2f} vs cold {itc.mean():.2f}")
