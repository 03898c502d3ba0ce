"""iwf_batch_solve: many independent problems with uneven windows in one call (the batched
sweep of potential strengths, phases and window cutoffs; every problem is Sec. 4.1's
eigenproblem). Each member is checked against the dense spectrum of its own oracle operator
and against a one-at-a-time solve of the same plan.
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


def _problems():
    # windows (K, L): three K = L sizes and two anisotropic ones, several potentials each
    eps, phases, _, _ = W.sweep_params(16, seed=4)
    shapes = [((2, 2), (2, 2)), ((3, 3), (3, 3)), ((2, 2), (2, 2)), ((3, 3), (2, 2)),
              ((4, 4), (2, 2)), ((3, 3), (3, 3)), ((2, 2), (3, 3))]
    out = []
    for i, (K, L) in enumerate(shapes):
        m, c = W.cosine_modes(4, eps[i], phases[i])
        out.append(W.Problem("sweep", W.moire_P(math.pi / 6), K, L, m, c))
    return out


@pytest.mark.parametrize("precision", ["f64", "c64"])
def test_batch_solve_uneven_windows_match_dense(iwf, precision):
    probs = _problems()
    plans = []
    for pb in probs:
        p = iwf.Plan(pb.P, pb.K, pb.L)
        p.set_potential(pb.modes, pb.coef)
        plans.append(p)
    assert len({p.N for p in plans}) >= 3
    nev, block = 4, 8
    ev, vecs, res, iters, info = iwf.batch_solve(plans, nev, block=block, precision=precision,
                                                 want_vectors=True)
    assert info["converged"] == 1 and np.max(res) <= 1e-10
    for q, (pb, p) in enumerate(zip(probs, plans)):
        win = O.build_window(pb.P, pb.K, pb.L)
        Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
        ref = O.eigen.dense_eigs(win, Vg, nev)[0]
        assert np.all(np.abs(ev[q] - ref) <= 1e-10 * np.maximum(1, np.abs(ref))), (q, ev[q], ref)
        X = vecs[q].cpu().numpy().T
        assert np.max(O.eigen.residual_norms(win, Vg, X, ev[q])) <= 2e-10
        one, _, _, _ = p.eigensolve(nev, block=block, precision=precision)
        assert np.all(np.abs(ev[q] - one) <= 1e-10 * np.maximum(1, np.abs(one)))
        assert iters[q] > 0


def test_batch_solve_rejects_non_separable_potentials(iwf):
    from paper_2404_04507_gb300 import capi
    pb = W.config_moire(eps=1.0, K=2, L=2)
    p = iwf.Plan(pb.P, pb.K, pb.L)
    # a mode on two lifted axes: V is kept as a full grid, not per-axis tables
    p.set_potential(np.array([[1, 1, 0, 0], [-1, -1, 0, 0]]), np.array([0.5, 0.5]))
    with pytest.raises(capi.IwfError) as e:
        iwf.batch_solve([p], 2, block=8)
    assert e.value.status == -10
