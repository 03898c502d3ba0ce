"""Pins of the oracle's irrational window and index-shift map (Sec. 3.1-3.2)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_04507_gb300 import workloads as W
from conftest import read_golden


def _golden():
    return {r[0]: int(r[1]) for r in read_golden("worked_window.txt")}


def test_worked_example_counts():
    g = _golden()
    P = np.array([[1.0, W.GOLDEN]])
    win = O.build_window(P, [g["K"]], [g["L"]])
    assert win.N == g["count_win"]
    assert win.lens == (g["kstar_I"], g["kstar_II"])
    box = O.build_window(P, [g["N_box"]], [g["N_box"]], method="pm")
    assert box.N == g["count_box"]


def test_worked_example_bijection_onto_hyperrectangle():
    P = np.array([[1.0, W.GOLDEN]])
    win = O.build_window(P, [2], [6])
    seen = {tuple(v) for v in win.kstar}
    assert len(seen) == 48
    assert seen == {(a, b) for a in range(4) for b in range(12)}


CASES = [
    (np.array([[1.0, W.GOLDEN]]), [2], [6]),
    (np.array([[1.0, math.sqrt(5.0)]]), [3], [5]),
    (2 * math.pi * np.array([[1.0, W.ALPHA_EX41]]), [4], [7]),
    (W.moire_P(math.pi / 6), [2, 3], [2, 2]),
    (W.random_P(2, 3, seed=7), [2, 2], [3]),
    (np.array([[1.3, 0.4, math.sqrt(2.0)], [-0.2, 0.9, math.sqrt(3.0)]]), [3, 2], [2]),
    (np.concatenate([np.eye(3), math.sqrt(2) * np.eye(3)], 1), [1, 2, 1], [1, 1, 2]),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("shift_round", [False, True])
@pytest.mark.parametrize("method", ["iwfpm", "pm"])
def test_two_step_inverse_equals_brute_force(case, shift_round, method):
    P, K, L = CASES[case]
    win = O.build_window(P, K, L, shift_round=shift_round, method=method)
    brute = O.brute_force_window(P, K, L, shift_round=shift_round, method=method)
    assert win.N == int(np.prod([2 * k for k in K]) * np.prod([2 * l for l in L]))
    assert brute.shape == win.k.shape
    assert np.array_equal(brute, win.k)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_map_is_mod_and_slices_are_runs(case):
    P, K, L = CASES[case]
    win = O.build_window(P, K, L)
    lens = np.asarray(win.lens)
    assert np.array_equal(win.kstar, np.mod(win.k, lens[None, :]))
    d = win.d
    # each k_II slice holds 2K_j consecutive integers per k_I axis, starting at lo_j
    per = int(np.prod(lens[:d]))
    for s in range(win.N // per):
        blk = win.k[s * per:(s + 1) * per]
        assert np.all(blk[:, d:] == blk[0, d:])
        for j in range(d):
            vals = np.unique(blk[:, j])
            assert vals.size == lens[j] and vals[-1] - vals[0] == lens[j] - 1


def test_window_order_is_lexicographic():
    win = O.build_window(W.moire_P(math.pi / 6), [2, 2], [2, 2])
    d = win.d
    key = [tuple(r[d:]) + tuple(r[:d]) for r in win.k.tolist()]
    assert key == sorted(key)


def test_exact_window_inequality_with_rational_ties():
    # moire P has Q entries 1/2, so (Q k_II)_j is an exact integer for some k_II:
    # the half-open interval then keeps exactly 2K points per slice.
    P = W.moire_P(math.pi / 6)
    win = O.build_window(P, [3, 3], [3, 3])
    Q = P[:, 2:]
    q = win.k[:, 2:].astype(float) @ Q.T
    v = win.k[:, :2] + q
    assert np.all(v >= -3 - 1e-12) and np.all(v < 3 + 1e-12)
    assert win.N == 6 * 6 * 6 * 6


def test_near_tie_is_rejected():
    P = np.array([[1.0, 0.5 + 1e-12]])
    with pytest.raises(O.WindowTie):
        O.build_window(P, [2], [3])


def test_rounded_shift_uses_half_away_from_zero():
    # Q = 1/2: k_II = +-1 gives q = +-1/2, rounded to +-1 (away from zero)
    P = np.array([[1.0, 0.5]])
    win = O.build_window(P, [2], [2], shift_round=True)
    for kII, lo in [(1, -3), (-1, -1), (-2, -1), (0, -2)]:
        kI = win.k[win.k[:, 1] == kII, 0]
        assert kI.min() == lo and kI.max() == lo + 3


def test_kinetic_diagonal():
    P = W.moire_P(0.3)
    win = O.build_window(P, [2, 2], [1, 1])
    for k, lam in zip(win.k[::7], win.lam[::7]):
        x = P @ k.astype(float)
        assert lam == pytest.approx(0.5 * float(x @ x), rel=1e-15, abs=1e-15)
