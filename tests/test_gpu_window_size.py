"""Window sizing from the decay of the coefficients (the "concentrated area" of the Fourier
coefficients, Sec. 4.2, Example 4.1): iwf_coef_extent against the window's definition, and
the sizing loop (accuracy.autosize) against a large-window reference.

A position k of the window K_{K,L} satisfies x_j = k_I,j + s_j in [-K_j, K_j) (s the index
shift, Sec. 3.2); a window of half-width K' with the same centring holds it exactly when
x_j in [-K', K'), i.e. K' >= max(ceil(-x_j), floor(x_j) + 1); along k_II, K' >= max(-k_II,j,
k_II,j + 1). The expected extents below are computed that way from the oracle's window.
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


def _expected_need(pb, k, mask):
    P = np.asarray(pb.P)
    d = P.shape[0]
    Q = np.zeros((d, P.shape[1] - d)) if pb.method == "pm" else O.split_Q(P)
    kI, kII = k[:, :d].astype(np.float64), k[:, d:]
    s = kII.astype(np.float64) @ Q.T if Q.shape[1] else np.zeros_like(kI)
    x = kI + s
    needI = np.maximum(np.ceil(-x), np.floor(x) + 1)
    needII = np.maximum(-kII, kII + 1)
    need = np.concatenate([needI, needII], axis=1)[mask]
    return need.max(axis=0).astype(np.int64) if need.size else np.zeros(k.shape[1], np.int64)


@pytest.mark.parametrize("pb", [W.example_41(2.5, 5, 20), W.example_41(2.5, 7, 12, method="pm"),
                                W.config_moire(eps=1.0, K=3, L=4)], ids=["ex41", "ex41_pm", "moire"])
def test_coef_extent_matches_window_geometry(iwf, pb):
    plan = iwf.Plan(pb.P, pb.K, pb.L, method=pb.method)
    win = O.build_window(pb.P, pb.K, pb.L, method=pb.method)
    k = win.k
    assert np.array_equal(plan.window().astype(np.int64), k)
    # coefficients decaying away from the window's centre, plus noise
    rng = np.random.default_rng(3)
    r = np.abs(k).sum(axis=1).astype(np.float64)
    c = np.exp(-0.4 * r) * (rng.standard_normal(win.N) + 1j * rng.standard_normal(win.N))
    ct = torch.from_numpy(c).cuda()
    for thr in (0.0, 1e-6, 1e-3, 1e-1, 10.0 * np.abs(c).max()):
        got = plan.coef_extent(ct, thr)
        want = _expected_need(pb, k, np.abs(c) >= thr)
        assert np.array_equal(got, want), (thr, got, want)
    # every point passes a zero threshold: the window's own half-widths
    assert np.array_equal(plan.coef_extent(ct, 0.0), np.array(list(pb.K) + list(pb.L)))


def test_autosize_example41_reaches_the_reference(iwf):
    # Example 4.1, v0 = 2.5 (extended state), started from a window too small in both K
    # and L; the sized window's ground state must agree with the large reference window
    from paper_2404_04507_gb300 import accuracy as A
    rounds = A.autosize(lambda K, L: W.example_41(2.5, K[0], L[0]), (2,), (12,), rel=1e-8)
    last = rounds[-1]
    assert last["fits"] and last["converged"] == 1 and len(rounds) > 1, rounds
    ref = A.ground_state(W.example_41(2.5, 5, 96))
    assert abs(last["E0"] - ref["E0"]) <= 1e-9 * abs(ref["E0"]), (rounds, ref["E0"])
    # the concentrated area is narrow in K (the paper's IWFPM windows use K = 5)
    assert last["need_K"][0] <= 6, rounds
