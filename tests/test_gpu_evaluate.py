"""GPU physical-space evaluation, normalisation, density and E_f against the oracle (Sec. 3.1
Eq. int; Sec. 4.2).

Tolerance of iwf_evaluate, derived from its arithmetic: each phase k.y is rounded with
relative error about eps, i.e. an absolute phase error of eps |theta|_max (theta = (P k).x);
Horner's rule along a row of l_f coefficients and the row-phase recurrence over l_s rows add
about (l_f + l_s) eps each. Every term has modulus |c_k|, so
|u_gpu - u_oracle| <= 16 eps (l_f + l_s + |theta|_max) sum|c| per point (the oracle's own
rounding is of the same form). A dropped slice, a wrong sign or a transposed P gives O(1).
The normalisation takes its integer decision (the first point of largest |u|^2) with the
same rounding on both sides, so the index must match exactly.
"""
import numpy as np
import pytest

import oracle as O
from oracle import transform as T
from paper_2404_04507_gb300 import workloads as W

from test_gpu_apply import PROBS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _setup(iwf, pb, seed=11):
    plan = iwf.Plan(pb.P, pb.K, pb.L, method=pb.method, shift_round=pb.shift_round)
    win = O.build_window(pb.P, pb.K, pb.L, shift_round=pb.shift_round, method=pb.method)
    c = W.random_block(win.N, 1, seed)[:, 0]
    return plan, win, c


def _tol(win, c, x):
    lf = win.lens[win.d - 1]
    ls = win.lens[win.d - 2] if win.d >= 2 else 1
    Pk = win.k.astype(np.float64) @ np.asarray(win.P).T
    theta = np.max(np.abs(x)) * np.max(np.sum(np.abs(Pk), axis=1))
    return 16 * EPS * (lf + ls + theta) * np.sum(np.abs(c))


def _gpu_eval(plan, c, x):
    u = plan.evaluate(torch.from_numpy(c).cuda(), torch.from_numpy(np.ascontiguousarray(x)).cuda())
    torch.cuda.synchronize()
    return u.cpu().numpy()


@pytest.mark.parametrize("name", sorted(PROBS))
@pytest.mark.parametrize("M", [7, 1000])
def test_evaluate_matches_oracle(iwf, name, M):
    pb = PROBS[name]
    plan, win, c = _setup(iwf, pb)
    x = np.random.default_rng(M).uniform(-50, 50, size=(M, win.d))
    got = _gpu_eval(plan, c, x)
    want = T.evaluate_quasi(win, c, x)
    assert np.max(np.abs(got - want)) <= _tol(win, c, x)


def test_evaluate_full_size_moire_on_the_paper_grid(iwf):
    # the 32^4 window, points from the first three rows of the 2D observation grid
    # [-50, 50]^2 (3003 points, ragged last tile), checked on a sample of 24 points
    pb = W.config_moire(eps=0.5)
    plan, win, c = _setup(iwf, pb)
    assert win.N == 32 ** 4
    x = W.physical_grid(2, rows=3)
    got = _gpu_eval(plan, c, x)
    pick = np.random.default_rng(5).choice(len(x), 24, replace=False)
    want = T.evaluate_quasi(win, c, x[pick])
    assert np.max(np.abs(got[pick] - want)) <= _tol(win, c, x)


def test_evaluate_many_points_single_group(iwf):
    # 320,000 points fill the GPU without slice groups (the kernel writes u directly)
    pb = PROBS["qse1d"]
    plan, win, c = _setup(iwf, pb)
    x = np.random.default_rng(2).uniform(-500, 500, size=(320_000, 1))
    got = _gpu_eval(plan, c, x)
    pick = np.random.default_rng(6).choice(len(x), 64, replace=False)
    pick = np.concatenate([pick, [0, len(x) - 1]])
    want = T.evaluate_quasi(win, c, x[pick])
    assert np.max(np.abs(got[pick] - want)) <= _tol(win, c, x)


def test_evaluate_is_deterministic_and_stream_ordered(iwf):
    pb = PROBS["moire_ragged"]
    plan, win, c = _setup(iwf, pb)
    ct = torch.from_numpy(c).cuda()
    xt = torch.from_numpy(np.random.default_rng(1).uniform(-50, 50, size=(513, 2))).cuda()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = plan.evaluate(ct, xt, stream=s)
        b = plan.evaluate(ct, xt, stream=s)
    s.synchronize()
    assert torch.equal(a, b)


def test_evaluate_argument_errors(iwf):
    from paper_2404_04507_gb300 import capi
    pb = PROBS["moire_small"]
    plan, win, c = _setup(iwf, pb)
    ct = torch.from_numpy(c).cuda()
    with pytest.raises(ValueError):
        plan.evaluate(ct, torch.zeros(4, 3, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        plan.evaluate(ct, torch.zeros(4, 2, dtype=torch.float32, device="cuda"))
    out = torch.full((1,), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    empty = torch.zeros(0, 2, dtype=torch.float64, device="cuda")
    plan.evaluate(ct, empty, out=out[:0])
    torch.cuda.synchronize()
    assert out[0].item() == 7.0 + 0j
    with pytest.raises(capi.IwfError):
        capi.check(capi.iwf_evaluate(plan.handle, None, None, 4, None, None), "iwf_evaluate")
    with pytest.raises(capi.IwfError):
        capi.check(capi.iwf_evaluate(plan.handle, ct.data_ptr(), empty.data_ptr(), -1,
                                     out.data_ptr(), None), "iwf_evaluate")
    with pytest.raises(capi.IwfError):
        capi.check(capi.iwf_field_normalize(plan.handle, None, 4, -1, None, None, None),
                   "iwf_field_normalize")
    z = torch.zeros(4, dtype=torch.complex128, device="cuda")
    with pytest.raises(capi.IwfError):
        plan.normalize_field(z, at=4)


def _random_field(M, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(M) + 1j * rng.standard_normal(M)


@pytest.mark.parametrize("M", [1, 1000, 300_001])
def test_normalize_matches_oracle(iwf, M):
    plan = iwf.Plan(PROBS["tiny"].P, (1,), (1,))
    u = _random_field(M, M)
    ut = torch.from_numpy(u).cuda()
    rho, idx = plan.normalize_field(ut)
    torch.cuda.synchronize()
    want, i = T.normalise_field(u)
    assert idx.item() == i
    assert np.max(np.abs(ut.cpu().numpy() - want)) <= 4 * EPS
    assert np.max(np.abs(rho.cpu().numpy() - T.density(want))) <= 8 * EPS


def test_normalize_ties_and_zero_field(iwf):
    plan = iwf.Plan(PROBS["tiny"].P, (1,), (1,))
    ut = torch.tensor([0.5, 2.0, -2.0, 2j, 2.0], dtype=torch.complex128, device="cuda")
    rho, idx = plan.normalize_field(ut)
    torch.cuda.synchronize()
    assert idx.item() == 1
    assert ut.cpu().numpy().tolist() == [0.25, 1.0, -1.0, 1j, 1.0]
    z = torch.zeros(300, dtype=torch.complex128, device="cuda")
    rho, idx = plan.normalize_field(z, want_rho=True)
    torch.cuda.synchronize()
    assert idx.item() == 0 and not torch.any(z) and not torch.any(rho)
    ut = torch.tensor([1.0, -2.0, 1j], dtype=torch.complex128, device="cuda")
    rho, idx = plan.normalize_field(ut, at=2)
    torch.cuda.synchronize()
    assert idx.item() == 2 and ut.cpu().numpy().tolist() == [-1j, 2j, 1.0]


def test_field_distance_matches_oracle(iwf):
    plan = iwf.Plan(PROBS["tiny"].P, (1,), (1,))
    u, v = _random_field(5001, 1), _random_field(5001, 2)
    d = plan.field_distance(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
    assert abs(d.item() - T.field_error(u, v)) <= 2 * EPS * T.field_error(u, v)
    e = torch.zeros(0, dtype=torch.complex128, device="cuda")
    assert plan.field_distance(e, e).item() == 0.0


@pytest.mark.parametrize("phases", [None, [0.3, 1.1]])
def test_ground_state_field_and_density_end_to_end(iwf, phases):
    # E_f of the 1D QSE ground state (eps = 3, window K = 12, L = 16) on the paper's grid
    # [-500, 500], h = 0.1: GPU solve -> GPU evaluate -> GPU normalise, against the dense
    # oracle eigenvector through the oracle's evaluation and normalisation. At residual 1e-10
    # and spectral gap 6.3e-3..6.7e-3 the vectors differ by about 1.5e-8 in 2-norm, i.e. a
    # few 1e-8 in the normalised field: the gate is 1e-6.
    # The even potential (no phases) has mirror twins of exactly equal |u| at +-279.6, where
    # u(-x) = conj(u(x)): rounding decides which one is the first largest, so the GPU's
    # choice is checked to be a maximum of the oracle's field and both are normalised at the
    # oracle's point. The phased potential has a unique maximum, which must match.
    pb = W.config_1d(K=12, L=16, eps=3.0)
    if phases is not None:
        m, c = W.cosine_modes(2, 3.0, phases)
        pb = W.Problem("qse1d_phased", pb.P, pb.K, pb.L, m, c)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    ev, X, res, info = plan.eigensolve(2, block=8, tol=1e-10)
    assert info["converged"] == 1
    x = W.physical_grid(1)
    u = plan.evaluate(X[0].contiguous(), torch.from_numpy(x).cuda())
    win = O.build_window(pb.P, pb.K, pb.L)
    Vg = O.grid_coefficients(pb.modes, pb.coef, win.lens)
    ref_ev, V = O.eigen.dense_eigs(win, Vg, 2)
    u_ref = T.evaluate_quasi(win, V[:, 0], x)
    want, i = T.normalise_field(u_ref)
    v = u.clone()
    rho, idx = plan.normalize_field(v)
    a = T.density(u_ref)
    assert a[idx.item()] >= a[i] * (1 - 1e-7)
    if phases is not None:
        assert idx.item() == i
    rho, _ = plan.normalize_field(u, at=i)
    ef = plan.field_distance(u, torch.from_numpy(want).cuda()).item()
    assert ef <= 1e-6, ef
    r = rho.cpu().numpy()
    assert abs(r.max() - 1.0) <= 1e-7 and abs(r[i] - 1.0) <= 4 * EPS
    assert np.max(np.abs(r - T.density(want))) <= 2e-6


GRID_PROBS = {
    "moire_small": PROBS["moire_small"],
    "moire_ragged": PROBS["moire_ragged"],
    "pm_moire": PROBS["pm_moire"],
    "ex42": W.example_42(0.8 * np.pi, 0.2 * np.pi, 6, 20),
    "random_grid_pot": PROBS["random_grid_pot"],
}


def _grid_points(origin, step, count):
    x0 = origin[0] + np.arange(count[0]) * step[0]
    x1 = origin[1] + np.arange(count[1]) * step[1]
    return np.ascontiguousarray(np.stack(np.meshgrid(x0, x1, indexing="ij"), -1).reshape(-1, 2))


@pytest.mark.parametrize("name", sorted(GRID_PROBS))
def test_evaluate_grid_matches_oracle(iwf, name):
    # a 70 x 130 grid: 2 x 3 tiles of 64 points, ragged in both directions
    pb = GRID_PROBS[name]
    plan, win, c = _setup(iwf, pb)
    origin, step, count = (-50.0, -50.0), (0.1, 0.1), (70, 130)
    got = plan.evaluate_grid(torch.from_numpy(c).cuda(), origin, step, count)
    torch.cuda.synchronize()
    x = _grid_points(origin, step, count)
    want = T.evaluate_quasi(win, c, x)
    assert np.max(np.abs(got.cpu().numpy() - want)) <= _tol(win, c, x)


def test_evaluate_grid_equals_direct_full_size(iwf):
    # the 32^4 window on 200 x 300 points of the 2D observation grid: the separable products
    # against direct summation, and the oracle on a sample
    pb = W.config_moire(eps=0.5)
    plan, win, c = _setup(iwf, pb)
    origin, step, count = (-50.0, -50.0), (0.1, 0.1), (200, 300)
    ct = torch.from_numpy(c).cuda()
    got = plan.evaluate_grid(ct, origin, step, count).cpu().numpy()
    x = _grid_points(origin, step, count)
    direct = plan.evaluate(ct, torch.from_numpy(x).cuda()).cpu().numpy()
    tol = _tol(win, c, x)
    assert np.max(np.abs(got - direct)) <= 2 * tol
    pick = np.random.default_rng(3).choice(len(x), 12, replace=False)
    assert np.max(np.abs(got[pick] - T.evaluate_quasi(win, c, x[pick]))) <= tol


def test_evaluate_grid_unsupported_and_empty(iwf):
    from paper_2404_04507_gb300 import capi
    skew = W.Problem("skew", np.array([[1.0, 0.3, 0.7], [0.2, 1.0, 0.5]]), (2, 2), (2,),
                     *W.cosine_modes(3, 1.0))
    for pb in (PROBS["qse1d"], skew, PROBS["qse3d_small"]):   # d = 1, P_I not diagonal, d = 3
        plan, win, c = _setup(iwf, pb)
        with pytest.raises(capi.IwfError) as e:
            plan.evaluate_grid(torch.from_numpy(c).cuda(), (0.0, 0.0), (0.1, 0.1), (4, 4))
        assert e.value.status == -10
    plan, win, c = _setup(iwf, PROBS["moire_small"])
    out = plan.evaluate_grid(torch.from_numpy(c).cuda(), (0.0, 0.0), (0.1, 0.1), (0, 7))
    assert out.numel() == 0
