"""Batched lockstep LOBPCG over problems sharing one geometry (the config-4 sweep form).

Each member of a batch must reproduce its own dense oracle spectrum to the FP64 tolerance
|lambda - lambda*| <= 1e-10 max(1, |lambda*|), and the same problem solved alone or inside a
batch must give the same eigenvalues.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_04507_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _dense(pb, nev):
    win = O.build_window(pb.P, pb.K, pb.L)
    Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
    return O.eigen.dense_eigs(win, Vg, nev)[0]


def _batch(K, params):
    probs = [W.config_moire(eps=e, K=K, L=K, phases=ph) for e, ph in params]
    return probs, [(pb.modes, pb.coef) for pb in probs]


@pytest.mark.parametrize("precision", ["f64", "c64"])
def test_batch_members_match_dense(iwf, precision):
    params = [(0.3, [0.1, 0.2, 0.3, 0.4]), (2.0, [1.0, 2.0, 3.0, 4.0]),
              (6.5, [5.0, 0.5, 2.5, 1.5]), (9.0, [0.0, 0.0, 0.0, 0.0])]
    probs, pots = _batch(3, params)
    plan = iwf.Plan(probs[0].P, probs[0].K, probs[0].L)
    ev, X, res, iters, info = plan.batch_eigensolve(pots, 8, block=12, precision=precision,
                                                    want_vectors=True)
    assert info["converged"] == 1
    for q, pb in enumerate(probs):
        ref = _dense(pb, 8)
        assert np.all(np.abs(ev[q] - ref) <= 1e-10 * np.maximum(1, np.abs(ref))), q
        assert np.max(res[q]) <= 1e-10 and iters[q] > 0
        Xq = X[q].cpu().numpy().T
        assert np.allclose(Xq.conj().T @ Xq, np.eye(8), atol=1e-12)


def test_batch_equals_single(iwf):
    params = [(1.5, [0.3, 0.7, 1.1, 2.9]), (4.0, [2.0, 0.4, 5.5, 3.3])]
    probs, pots = _batch(4, params)
    plan = iwf.Plan(probs[0].P, probs[0].K, probs[0].L)
    evb, _, _, _, _ = plan.batch_eigensolve(pots, 6, block=10)
    for q, pb in enumerate(probs):
        single = iwf.Plan(pb.P, pb.K, pb.L)
        single.set_potential(pb.modes, pb.coef)
        ev, _, _, _ = single.eigensolve(6, block=10)
        assert np.allclose(evb[q], ev, rtol=1e-10, atol=1e-10)


def test_sweep_group_residual_certificate(iwf):
    # two problems of the config-4 distribution that share K = L
    eps, phases, cut, KL = W.sweep_params(64, seed=4)
    k = int(np.min(KL))
    idx = [i for i in range(64) if KL[i] == k][:2]
    probs = [W.sweep_problem(eps[i], phases[i], KL[i]) for i in idx]
    plan = iwf.Plan(probs[0].P, probs[0].K, probs[0].L)
    ev, X, res, iters, info = plan.batch_eigensolve([(p.modes, p.coef) for p in probs], 16,
                                                    block=24, want_vectors=True)
    assert info["converged"] == 1
    for q, pb in enumerate(probs):
        win = O.build_window(pb.P, pb.K, pb.L)
        Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
        Xq = X[q].cpu().numpy().T
        assert np.max(O.eigen.residual_norms(win, Vg, Xq[:, :4], ev[q, :4])) <= 2e-10


def test_batch_rejects_multi_axis_modes(iwf):
    from paper_2404_04507_gb300 import capi
    pb = W.config_moire(eps=1.0, K=3, L=3)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    m = np.array([[1, 1, 0, 0], [-1, -1, 0, 0]])
    c = np.array([0.5, 0.5], dtype=complex)
    with pytest.raises(capi.IwfError) as e:
        plan.batch_eigensolve([(m, c)], 4, block=4)
    assert e.value.status == -10


@pytest.mark.parametrize("precision", ["f64", "c64"])
def test_batch_on_pencil_path(iwf, precision):
    # K = L = 8 (16^4 grid) runs the pencil kernels: per-problem potential tables and skipped
    # converged problems inside them; the tiled kernels on the same batch give the same
    # eigenvalues and the oracle certifies the residuals
    params = [(0.7, [0.2, 1.4, 2.2, 0.9]), (5.0, [3.0, 0.3, 4.1, 1.7])]
    probs, pots = _batch(8, params)
    plan = iwf.Plan(probs[0].P, probs[0].K, probs[0].L)
    assert plan.schedule(precision)["path"] == "pencil"
    ev, X, res, iters, info = plan.batch_eigensolve(pots, 4, block=8, precision=precision,
                                                    want_vectors=True)
    assert info["converged"] == 1
    plan.set_path("f64", "tiled")
    plan.set_path("c64", "tiled")
    ev_t, _, _, _, _ = plan.batch_eigensolve(pots, 4, block=8, precision=precision)
    assert np.allclose(ev, ev_t, rtol=1e-10, atol=1e-10)
    for q, pb in enumerate(probs):
        win = O.build_window(pb.P, pb.K, pb.L)
        Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
        Xq = X[q].cpu().numpy().T
        assert np.max(O.eigen.residual_norms(win, Vg, Xq, ev[q])) <= 2e-10
