"""GPU parity of the window, the kinetic diagonal and H~ psi against the CPU oracle.

Tolerances: window and slice bounds are integer work and must match bit for bit. The
FP64 apply is compared element-wise with |err| <= 1e-12 max|H psi|: two FFT passes of
length <= 2^20 contribute O(log2 N * 2^-53) relative error, far below that bound, while a
dropped term, sign or index error is O(1). The complex64 apply is held to 2e-5 max|H psi|
(same argument with 2^-24).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2404_04507_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 2e-5


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _plan(iwf, pb, shift_round=False):
    plan = iwf.Plan(pb.P, pb.K, pb.L, method=pb.method, shift_round=shift_round)
    plan.set_potential(pb.modes, pb.coef)
    return plan


def _oracle(pb, shift_round=False):
    win = O.build_window(pb.P, pb.K, pb.L, shift_round=shift_round, method=pb.method)
    return win, O.grid_coefficients(pb.modes, pb.coef, win.lens)


def _gpu_apply(plan, X, dtype):
    xt = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype).cuda()
    y = plan.apply(xt)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.complex128).T


def _problems():
    P3 = np.concatenate([np.eye(3), math.sqrt(2) * np.eye(3)], 1)
    m3, c3 = W.cosine_modes(6, 3.0)
    mr, cr = W.random_modes(3, 5, 3, seed=5)
    return {
        "qse1d": W.config_1d(),
        "moire_small": W.config_moire(eps=5.0, K=3, L=4),
        "moire_ragged": W.config_moire(eps=0.5, K=5, L=3, phases=[0.3, 1.1, 2.0, 4.0]),
        "pm_moire": W.config_moire(eps=0.5, K=4, L=4, method="pm"),
        "qse3d_small": W.Problem("qse3d_small", P3, (2, 2, 1), (1, 2, 2), m3, c3),
        "random_grid_pot": W.Problem("rnd", W.random_P(2, 3, seed=2), (3, 4), (5,), mr, cr),
        "ex41_round": W.example_41(2.5, 6, 13, shift_round=True),
        "tiny": W.Problem("tiny", np.array([[1.0, math.sqrt(3.0)]]), (1,), (1,),
                          *W.cosine_modes(2, 1.0)),
    }


PROBS = _problems()


@pytest.mark.parametrize("name", list(PROBS))
def test_window_bit_exact(iwf, name):
    pb = PROBS[name]
    rnd = pb.shift_round
    plan = _plan(iwf, pb, rnd)
    win, _ = _oracle(pb, rnd)
    assert plan.N == win.N
    assert np.array_equal(plan.window().astype(np.int64), win.k)
    assert np.allclose(plan.kinetic(), win.lam, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_apply_matches_oracle(iwf, name, prec):
    pb = PROBS[name]
    plan = _plan(iwf, pb, pb.shift_round)
    win, Vg = _oracle(pb, pb.shift_round)
    X = W.random_block(win.N, 3, seed=11)
    want = O.apply_stencil(win, Vg, X)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    got = _gpu_apply(plan, X.astype(np.complex64) if prec == "c64" else X, dtype)
    if prec == "c64":
        want = O.apply_stencil(win, Vg, X.astype(np.complex64).astype(np.complex128))
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_window_full_size_moire(iwf):
    pb = W.config_moire(eps=0.5)
    plan = _plan(iwf, pb)
    win, _ = _oracle(pb)
    assert plan.N == 32 ** 4 == win.N
    assert np.array_equal(plan.window().astype(np.int64), win.k)


def test_apply_full_size_moire_block(iwf):
    # the benchmarked launch: 16 vectors of the 32^4 grid, FP64; the oracle checks 2 of them
    pb = W.config_moire(eps=5.0)
    plan = _plan(iwf, pb)
    win, Vg = _oracle(pb)
    X = W.random_block(win.N, 16, seed=3)
    got = _gpu_apply(plan, X, torch.complex128)
    for c in (0, 15):
        want = O.apply_stencil(win, Vg, X[:, c])
        assert np.max(np.abs(got[:, c] - want)) <= TOL64 * np.max(np.abs(want))


def test_hermitian_on_gpu(iwf):
    pb = W.config_moire(eps=0.5, K=6, L=5)
    plan = _plan(iwf, pb)
    N = plan.N
    X = W.random_block(N, 2, seed=9)
    HX = _gpu_apply(plan, X, torch.complex128)
    lhs = np.vdot(X[:, 0], HX[:, 1])
    rhs = np.vdot(HX[:, 0], X[:, 1])
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_empty_block_is_noop(iwf):
    plan = _plan(iwf, PROBS["tiny"])
    x = torch.zeros((0, plan.N), dtype=torch.complex128, device="cuda")
    plan.apply(x)


def test_errors_are_reported(iwf):
    from paper_2404_04507_gb300 import capi
    with pytest.raises(capi.IwfError) as e:
        iwf.Plan(np.array([[1.0, 0.5 + 1e-12]]), [2], [3])
    assert e.value.status == -9
    with pytest.raises(capi.IwfError) as e:
        iwf.Plan(np.array([[1.0, 2.0 ** 0.5]]), [17], [3])
    assert e.value.status == -10
    plan = iwf.Plan(np.array([[1.0, 2.0 ** 0.5]]), [2], [3])
    x = torch.zeros(plan.N, dtype=torch.complex128, device="cuda")
    with pytest.raises(capi.IwfError) as e:
        plan.apply(x)
    assert e.value.status == -1
    with pytest.raises(capi.IwfError) as e:
        plan.set_potential(np.array([[1, 0]]), np.array([1.0 + 0j]))   # not real
    assert e.value.status == -1


@pytest.mark.parametrize("sched", [(128, 24, 24), (128, 96, 48), (256, 48, 96), (256, 160, 48)])
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_every_schedule_gives_the_same_operator(iwf, sched, prec):
    pb = PROBS["moire_ragged"]
    plan = _plan(iwf, pb)
    plan.set_schedule(prec, *sched)
    win, Vg = _oracle(pb)
    X = W.random_block(win.N, 5, seed=12)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    Xin = X.astype(np.complex64).astype(np.complex128) if prec == "c64" else X
    got = _gpu_apply(plan, Xin, dtype)
    want = O.apply_stencil(win, Vg, Xin)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_autotune_picks_a_valid_schedule(iwf):
    pb = W.config_moire(eps=0.5, K=8, L=8)
    plan = _plan(iwf, pb)
    ms, best = plan.autotune("c64", nvec=4)
    sched = plan.schedule("c64")
    assert ms > 0 and best[2] in (12, 24, 48, 96) and sched["chunk_mb"] == best[2]
    if sched["path"] == "pencil":
        assert best[:2] == (0, 0)
    else:
        assert best[0] in (128, 256) and best[1] in (24, 48, 96, 160)
    win, Vg = _oracle(pb)
    X = W.random_block(win.N, 2, seed=1).astype(np.complex64).astype(np.complex128)
    got = _gpu_apply(plan, X, torch.complex64)
    want = O.apply_stencil(win, Vg, X)
    assert np.max(np.abs(got - want)) <= TOL32 * np.max(np.abs(want))


# The pencil path: n = 4, d = 2, two equal k_I axis lengths and two equal k_II axis lengths,
# each 16 or 32 (the moire family). Same tolerances as the tiled path.
PENCIL = {
    "moire16": W.config_moire(eps=0.5, K=8, L=8),
    "moire16_phases": W.config_moire(eps=5.0, K=8, L=8, phases=[0.3, 1.1, 2.0, 4.0]),
    "moire_kI16_kII32": W.config_moire(eps=0.5, K=8, L=16),
    "moire_kI32_kII16": W.config_moire(eps=2.0, K=16, L=8, phases=[2.0, 0.1, 1.3, 5.9]),
    # multi-axis modes: the potential is a full grid, not per-axis tables
    "grid_pot": W.Problem("rnd4", W.random_P(2, 4, seed=7), (8, 8), (8, 8),
                          *W.random_modes(4, 6, 3, seed=8)),
}


@pytest.mark.parametrize("name", list(PENCIL))
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_pencil_path_matches_oracle(iwf, name, prec):
    pb = PENCIL[name]
    plan = _plan(iwf, pb)
    assert plan.schedule(prec)["path"] == "pencil"
    win, Vg = _oracle(pb)
    X = W.random_block(win.N, 3, seed=21)
    if prec == "c64":
        X = X.astype(np.complex64).astype(np.complex128)
    got = _gpu_apply(plan, X, torch.complex128 if prec == "f64" else torch.complex64)
    want = O.apply_stencil(win, Vg, X)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_pencil_and_tiled_paths_agree_full_size(iwf, prec):
    # the benchmarked 16-vector block of the 32^4 grid through both kernel sets, with the
    # oracle on two vectors; chunks of 2 vectors make the pencil path loop over chunks
    pb = W.config_moire(eps=5.0)
    plan = _plan(iwf, pb)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    X = W.random_block(plan.N, 16, seed=5)
    if prec == "c64":
        X = X.astype(np.complex64).astype(np.complex128)
    plan.set_schedule(prec, 128, 96, 16 if prec == "c64" else 32)
    got_p = _gpu_apply(plan, X, dtype)
    plan.set_path(prec, "tiled")
    got_t = _gpu_apply(plan, X, dtype)
    tol = TOL64 if prec == "f64" else TOL32
    scale = np.max(np.abs(got_t))
    assert np.max(np.abs(got_p - got_t)) <= 2 * tol * scale
    win, Vg = _oracle(pb)
    for c in (0, 15):
        want = O.apply_stencil(win, Vg, X[:, c])
        assert np.max(np.abs(got_p[:, c] - want)) <= tol * np.max(np.abs(want))


# Double-float DFTs of an FP64 apply (IWF_ARITH_DF): storage, potential and kinetic term stay
# FP64, the DFTs carry about 48 bits; same element-wise tolerance as the FP64 path.
@pytest.mark.parametrize("name", list(PENCIL))
def test_double_float_dfts_match_oracle(iwf, name):
    pb = PENCIL[name]
    plan = _plan(iwf, pb)
    plan.set_arith("df")
    win, Vg = _oracle(pb)
    X = W.random_block(win.N, 3, seed=22)
    X[:, 1] *= 10.0 ** np.random.default_rng(4).uniform(-40, 0, size=win.N)   # wide range
    got = _gpu_apply(plan, X, torch.complex128)
    want = O.apply_stencil(win, Vg, X)
    for c in range(3):
        err = np.max(np.abs(got[:, c] - want[:, c])) / np.max(np.abs(want[:, c]))
        assert err <= TOL64, (c, err)


@pytest.mark.parametrize("eps", [0.5, 5.0])
def test_double_float_dfts_full_size(iwf, eps):
    pb = W.config_moire(eps=eps)
    plan = _plan(iwf, pb)
    X = W.random_block(plan.N, 16, seed=6)
    got64 = _gpu_apply(plan, X, torch.complex128)
    plan.set_arith("df")
    gotdf = _gpu_apply(plan, X, torch.complex128)
    assert np.max(np.abs(gotdf - got64)) <= TOL64 * np.max(np.abs(got64))
    plan.set_arith("f64")
    assert np.array_equal(_gpu_apply(plan, X[:, :2], torch.complex128), got64[:, :2])


def test_double_float_dfts_need_the_pencil_path(iwf):
    from paper_2404_04507_gb300 import capi
    plan = _plan(iwf, PROBS["moire_ragged"])
    with pytest.raises(capi.IwfError) as e:
        plan.set_arith("df")
    assert e.value.status == -10
    plan = _plan(iwf, PENCIL["moire16"])
    plan.set_arith("df")
    with pytest.raises(capi.IwfError) as e:
        plan.set_path("f64", "tiled")
    assert e.value.status == -10
    plan.set_arith("f64")
    plan.set_path("f64", "tiled")
    with pytest.raises(capi.IwfError) as e:
        plan.set_arith("df")
    assert e.value.status == -10


def test_path_selection(iwf):
    from paper_2404_04507_gb300 import capi
    plan = _plan(iwf, PROBS["moire_ragged"])
    assert plan.schedule("f64")["path"] == "tiled"
    with pytest.raises(capi.IwfError) as e:
        plan.set_path("f64", "pencil")
    assert e.value.status == -10
    plan = _plan(iwf, PENCIL["moire16"])
    plan.set_path("c64", "tiled")
    assert plan.schedule("c64")["path"] == "tiled"
    assert plan.schedule("f64")["path"] == "pencil"
    plan.set_path("c64", "auto")
    assert plan.schedule("c64")["path"] == "pencil"


def test_overlapping_blocks_are_rejected(iwf):
    from paper_2404_04507_gb300 import capi
    pb = PENCIL["moire16"]
    plan = _plan(iwf, pb)
    x = torch.zeros((3, plan.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.IwfError) as e:
        plan.apply(x, x)
    assert e.value.status == -1
    with pytest.raises(capi.IwfError) as e:
        plan.apply(x[:2], x[1:])                      # shifted by one vector
    assert e.value.status == -1


@pytest.mark.parametrize("prec", ["f64", "c64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_matches_device_apply(iwf, prec, pinned):
    # iwf_apply_host pipelines chunks of the block through the device; its result must equal
    # iwf_apply's on the same vectors (same kernels), for 7 vectors in chunks of 2, 2, 2, 1
    pb = PENCIL["moire16"]
    plan = _plan(iwf, pb)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    X = W.random_block(plan.N, 7, seed=8)
    xh = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype)
    if pinned:
        xh = xh.pin_memory()
    yh = plan.apply_host(xh)
    yd = plan.apply(xh.cuda()).cpu()
    assert torch.equal(yh, yd)
    win, Vg = _oracle(pb)
    Xin = xh.numpy().T.astype(np.complex128)
    want = O.apply_stencil(win, Vg, Xin[:, 6])
    tol = TOL64 if prec == "f64" else TOL32
    got = yh.numpy().T[:, 6].astype(np.complex128)
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_apply_host_rejects_bad_arguments(iwf):
    from paper_2404_04507_gb300 import capi
    plan = _plan(iwf, PENCIL["moire16"])
    x = torch.zeros((2, plan.N), dtype=torch.complex128)
    with pytest.raises(capi.IwfError) as e:
        plan.apply_host(x, x)
    assert e.value.status == -1
    with pytest.raises(TypeError):
        plan.apply_host(x.cuda())


# Direct-convolution apply (the ablation of the FFT passes): same operator, every shape.
@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_stencil_apply_matches_oracle(iwf, name, prec):
    pb = PROBS[name]
    plan = _plan(iwf, pb, pb.shift_round)
    win, Vg = _oracle(pb, pb.shift_round)
    X = W.random_block(win.N, 3, seed=31)
    if prec == "c64":
        X = X.astype(np.complex64).astype(np.complex128)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    xt = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype).cuda()
    got = plan.apply_stencil(xt).cpu().numpy().astype(np.complex128).T
    want = O.apply_stencil(win, Vg, X)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_stencil_and_fft_apply_agree_full_size(iwf, prec):
    pb = W.config_moire(eps=5.0, phases=[0.4, 1.9, 3.3, 5.0])
    plan = _plan(iwf, pb)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    x = torch.from_numpy(np.ascontiguousarray(W.random_block(plan.N, 4, seed=2).T)).to(dtype).cuda()
    a = plan.apply(x)
    b = plan.apply_stencil(x)
    tol = TOL64 if prec == "f64" else TOL32
    assert float((a - b).abs().max()) <= 2 * tol * float(a.abs().max())


# axes longer than the register codelets (32): the tiled passes run a shared-memory
# mixed-radix FFT on every axis of such a group
LONG = {
    "qse1d_L20": W.config_1d(K=5, L=20),                              # 10 x 40 (4 2 5)
    "ex41_L60": W.example_41(2.5, 5, 60),                             # 10 x 120 (4 2 3 5)
    "pm_both_long": W.config_1d(K=24, L=64, method="pm"),             # 48 x 128
    "moire_L20": W.config_moire(eps=0.5, K=3, L=20),                  # 6^2 x 40^2
    "radix7_round": W.Problem("r7", np.array([[1.0, math.sqrt(7.0)]]), (21,), (3,),
                              *W.cosine_modes(2, 1.5), shift_round=True),   # 42 (2 3 7) x 6
}


@pytest.mark.parametrize("name", list(LONG))
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_long_axes_match_oracle(iwf, name, prec):
    pb = LONG[name]
    plan = _plan(iwf, pb, pb.shift_round)
    win, Vg = _oracle(pb, pb.shift_round)
    assert np.array_equal(plan.window().astype(np.int64), win.k)
    X = W.random_block(win.N, 3, seed=12)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    got = _gpu_apply(plan, X.astype(np.complex64) if prec == "c64" else X, dtype)
    want = O.apply_stencil(win, Vg, X.astype(np.complex64).astype(np.complex128)
                           if prec == "c64" else X)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


# k_II groups above 8192 points (one shared-memory tile): pass B runs as one pass per k_II
# axis, the multiply by V in the last one (Example 4.3 from L = 20 needs this)
SPLIT = {
    "three_axes_24": W.Problem("s3", np.array([[1.0, 2.0 ** 0.5, 3.0 ** 0.5, 5.0 ** 0.5]]),
                               (2,), (12, 12, 12), *W.cosine_modes(4, 1.5)),   # 4 x 24^3
    "long_axes": W.Problem("sl", np.array([[1.0, 2.0 ** 0.5, 3.0 ** 0.5]]), (3,), (64, 40),
                           *W.cosine_modes(3, 0.7)),                          # 6 x 128 x 80
    "grid_potential": W.Problem("sg", W.random_P(1, 4, seed=3), (2,), (12, 12, 12),
                                *W.random_modes(4, 6, 2, seed=7)),             # full-grid V
    "ex43_K2_L12": W.example_43(math.pi, K=2, L=12),                          # 4^3 x 24^3
}


@pytest.mark.parametrize("name", list(SPLIT))
@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_split_k2_group_matches_oracle(iwf, name, prec):
    pb = SPLIT[name]
    plan = _plan(iwf, pb)
    win, Vg = _oracle(pb)
    assert int(np.prod([2 * l for l in pb.L])) > 8192
    assert np.array_equal(plan.window().astype(np.int64), win.k)
    X = W.random_block(win.N, 2, seed=21)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    got = _gpu_apply(plan, X.astype(np.complex64) if prec == "c64" else X, dtype)
    want = O.apply_stencil(win, Vg, X.astype(np.complex64).astype(np.complex128)
                           if prec == "c64" else X)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("prec", ["f64", "c64"])
def test_longest_axis_full_size(iwf, prec):
    # 2L = 8192 (L = 4096, the paper's largest 1D window): one k_II group of 8192 points, the
    # most a tile holds; 4 vectors, all checked
    pb = W.config_1d(K=5, L=4096)
    plan = _plan(iwf, pb)
    win, Vg = _oracle(pb)
    assert plan.N == 10 * 8192
    X = W.random_block(win.N, 4, seed=13)
    dtype = torch.complex128 if prec == "f64" else torch.complex64
    got = _gpu_apply(plan, X.astype(np.complex64) if prec == "c64" else X, dtype)
    want = O.apply_stencil(win, Vg, X.astype(np.complex64).astype(np.complex128)
                           if prec == "c64" else X)
    tol = TOL64 if prec == "f64" else TOL32
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_long_axis_limits(iwf):
    from paper_2404_04507_gb300 import capi
    for K in (17, 4097, 11 * 4):          # 34 = 2 x 17, 8194 > 8192, 88 = 8 x 11
        with pytest.raises(capi.IwfError) as e:
            iwf.Plan(np.array([[1.0, 2.0 ** 0.5]]), [K], [3])
        assert e.value.status == -10


@pytest.mark.parametrize("precision", ["f64", "c64"])
def test_long_axis_eigensolve_matches_dense(iwf, precision):
    # Example 4.1 at the paper's K = 5, L = 60 (10 x 120 grid): the solver on the long kernels
    pb = W.example_41(2.5, 5, 60)
    plan = _plan(iwf, pb)
    win, Vg = _oracle(pb)
    ev, X, res, info = plan.eigensolve(6, block=8, tol=1e-10, precision=precision)
    ref = O.eigen.dense_eigs(win, Vg, 6)[0]
    assert info["converged"] == 1
    assert np.all(np.abs(ev - ref) <= 1e-10 * np.maximum(1.0, np.abs(ref))), np.max(np.abs(ev - ref))
