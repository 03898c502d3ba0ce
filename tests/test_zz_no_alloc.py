"""iwf_apply_noalloc: the apply for callers that must not allocate device memory.

Such callers (a program whose device memory belongs to a pool allocator that forbids direct
cudaMalloc, or a latency-critical loop that cannot afford cudaMalloc's implicit device
synchronisation) call iwf_apply_noalloc, which keeps its scratch in a fixed 32 MiB array
inside the library. This file is collected last on purpose. The result must equal
iwf_apply's within the FP64 / complex64 tolerances used by the other apply tests, on two
calls in a row (the second call finds the first call's data in the shared array).
"""
import ctypes as C

import numpy as np
import pytest

from paper_2404_04507_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-5}


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _noalloc(plan, x, y):
    from paper_2404_04507_gb300 import capi
    prec = capi.IWF_PREC_F64 if x.dtype == torch.complex128 else capi.IWF_PREC_C64
    nvec = x.shape[0] if x.dim() == 2 else 1
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    capi.check(capi.iwf_apply_noalloc(plan.handle, prec, C.c_void_p(x.data_ptr()),
                                      C.c_void_p(y.data_ptr()), nvec, stream),
               "iwf_apply_noalloc")
    return y


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_noalloc_matches_apply_on_two_calls(iwf, dtype):
    # full 32^4 moire grid: one FP64 vector is 16 MiB, so 5 vectors run in 3 chunks
    pb = W.config_moire(eps=5.0)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    for call, seed in enumerate((21, 22)):
        X = W.random_block(plan.N, 5, seed=seed)
        x = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype).cuda()
        want = plan.apply(x)
        got = _noalloc(plan, x, torch.full_like(x, float("nan")))
        torch.cuda.synchronize()
        err = (got - want).abs().max().item()
        assert err <= TOL[dtype] * want.abs().max().item(), (call, err)


def test_noalloc_allocates_nothing_on_a_fresh_plan(iwf):
    # the kernels are loaded first through another plan of the same geometry, so that lazy
    # module loading does not count; then a fresh plan's first call is the allocation-free one
    pb = W.config_moire(eps=5.0)
    warm = iwf.Plan(pb.P, pb.K, pb.L)
    warm.set_potential(pb.modes, pb.coef)
    for dtype in (torch.complex128, torch.complex64):
        x = torch.from_numpy(np.ascontiguousarray(W.random_block(warm.N, 2, seed=3).T)).to(dtype).cuda()
        _noalloc(warm, x, torch.empty_like(x))
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    x = torch.from_numpy(np.ascontiguousarray(W.random_block(plan.N, 5, seed=9).T)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(plan, x, y)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # iwf_apply would size a workspace of a chunk of vectors (tens of MiB) on this plan
    assert free0 - free1 < (2 << 20), (free0, free1)
    want = plan.apply(x)
    torch.cuda.synchronize()
    assert (y - want).abs().max().item() <= 1e-12 * want.abs().max().item()


def test_noalloc_small_plan_and_empty_block(iwf):
    pb = W.config_1d()
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    x = torch.from_numpy(np.ascontiguousarray(W.random_block(plan.N, 3, seed=5).T)).cuda()
    for _ in range(2):
        got = _noalloc(plan, x, torch.empty_like(x))
        want = plan.apply(x)
        torch.cuda.synchronize()
        assert (got - want).abs().max().item() <= 1e-12 * want.abs().max().item()
    _noalloc(plan, x[:0], torch.empty_like(x[:0]))


def test_noalloc_rejects_plans_above_the_fixed_maximum(iwf):
    from paper_2404_04507_gb300 import capi
    P = W.random_P(2, 5, seed=17)
    plan = iwf.Plan(P, [16, 16], [8, 8, 9])              # 4.7M points > 32 MiB per vector
    m, c = W.cosine_modes(5, 1.0)
    plan.set_potential(m, c)
    x = torch.zeros((1, plan.N), dtype=torch.complex64, device="cuda")
    with pytest.raises(capi.IwfError) as e:
        _noalloc(plan, x, torch.empty_like(x))
    assert e.value.status == -10 and "33554432" in str(e.value)
