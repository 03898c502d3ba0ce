"""Failure paths of the C ABI: non-finite inputs and a bounded device wait that runs out.

Nothing here faults or hangs the GPU. Non-finite values are planted on the host (a NaN in a
potential coefficient, in the start block X0). The timeout is made deterministic by the plan's
wait-limit knob: with a limit of 0 rounds every pipelined pass C (complex-float pencil path)
gives up at its first wait, drains the copies it already issued with the full bound, records
IWF_ERR_TIMEOUT in the plan's device error word and returns; the host reads the word at the
plan's next synchronisation point.
"""
import numpy as np
import pytest

from paper_2404_04507_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT, NONFINITE = -8, -5


@pytest.fixture(scope="module")
def iwf():
    import paper_2404_04507_gb300 as iwf
    assert torch.cuda.is_available()
    return iwf


def _moire16(iwf):
    pb = W.config_moire(eps=0.5, K=8, L=8)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    plan.set_path("c64", "pencil")
    return plan


def _block(plan, nvec, seed, dtype=torch.complex64):
    X = W.random_block(plan.N, nvec, seed=seed)
    return torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype).cuda()


def test_nan_in_potential_is_rejected(iwf):
    from paper_2404_04507_gb300 import capi
    pb = W.config_moire(eps=0.5, K=8, L=8)
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    coef = pb.coef.copy()
    coef[1] = complex(np.nan, 0.0)
    with pytest.raises(capi.IwfError) as e:
        plan.set_potential(pb.modes, coef)
    assert e.value.status == NONFINITE


@pytest.mark.parametrize("precision", ["f64", "c64"])
def test_nan_in_start_block_is_reported(iwf, precision):
    from paper_2404_04507_gb300 import capi
    pb = W.config_1d()
    plan = iwf.Plan(pb.P, pb.K, pb.L)
    plan.set_potential(pb.modes, pb.coef)
    X0 = _block(plan, 8, seed=4, dtype=torch.complex128)
    X0[3, 17] = complex(float("nan"), 0.0)
    with pytest.raises(capi.IwfError) as e:
        plan.eigensolve(8, block=8, precision=precision, X0=X0, maxit=50)
    assert e.value.status == NONFINITE


def test_wait_timeout_is_reported_then_cleared(iwf):
    from paper_2404_04507_gb300 import capi
    plan = _moire16(iwf)
    x = _block(plan, 4, seed=7)
    want = plan.apply(x)
    plan.check()                                   # nothing pending
    plan.set_wait_limit(0)
    plan.apply(x, out=torch.zeros_like(x))         # enqueues; the error shows at the check
    with pytest.raises(capi.IwfError) as e:
        plan.check()
    assert e.value.status == TIMEOUT
    plan.check()                                   # the word was cleared
    plan.set_wait_limit(-1)
    got = plan.apply(x)
    plan.check()
    err = (got - want).abs().max().item()
    assert err <= 2e-5 * want.abs().max().item()


def test_wait_timeout_reaches_the_synchronous_calls(iwf):
    from paper_2404_04507_gb300 import capi
    plan = _moire16(iwf)
    plan.set_wait_limit(0)
    xh = _block(plan, 3, seed=8).cpu().pin_memory()
    with pytest.raises(capi.IwfError) as e:
        plan.apply_host(xh)
    assert e.value.status == TIMEOUT
    with pytest.raises(capi.IwfError) as e:
        plan.eigensolve(4, block=8, precision="c64", maxit=20)
    assert e.value.status == TIMEOUT
    plan.set_wait_limit(-1)
    plan.check()
    ev, _, res, info = plan.eigensolve(4, block=8, precision="c64", tol=1e-8)
    assert info["converged"] == 1 and np.all(res <= 1e-8)
