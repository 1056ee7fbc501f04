"""Failure paths and accounting of the GPU library, through the C ABI.

* A Newton-Schulz step that does not reduce the residual (eq. newton needs
  the spectral radius of I - A X below 1) ends the tail and leaves the
  better iterate from before it, as the oracle's ns_diverged exit does.
* The bounded device-side waits of the tcgen05 kernels: a self-test launch
  whose loads are never issued must come back as IBMI_ERR_TIMEOUT, with the
  CUDA context still usable (no fault, no hang).
* The flops a result reports follow the Section 4 cost model the oracle
  counts (plan_flops, sweep_flops) plus 2 p^3 per residual.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ibmi_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibmi():
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as m
    return m


def test_fp64_tail_divergence_keeps_the_handover_iterate(ibmi):
    """KMS, two sets, initial guess 100 I: one sweep leaves ||I - A H|| far
    above 1, the step grows it; like the oracle, H is the hand-over iterate."""
    p, rho = 16, 0.9
    A = wl.kms(p, rho)
    h0 = 100.0 * np.eye(p)
    ref = O.ibmi(A, O.partition(p, 2, 0), tol=1e-12, max_sweeps=50, ns_theta=1e9, h0=h0)
    assert ref.status == "ns_diverged"
    dA = torch.from_numpy(A).cuda()
    dH = torch.from_numpy(h0.copy()).cuda()
    plan = ibmi.ibmi_plan(p, K=2, h=0, tol=1e-12, max_sweeps=50, ns_theta=1e9, init=ibmi.IBMI_INIT_USER)
    s, res = ibmi.ibmi_invert(plan, dA, dH)
    plan.close()
    H = dH.cpu().numpy()
    assert s == ibmi.IBMI_NOT_CONVERGED and res["sweeps"] == 1 and res["ns_steps"] == 1, res
    assert np.abs(H - ref.h).max() <= 1e-12 * np.abs(ref.h).max()
    assert res["resid_f"] == pytest.approx(ref.resid_f, rel=1e-12)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refine_divergence_restores_the_input(ibmi, precision):
    """X_0 = 3 A^{-1}: I - A X_0 = -2 I, the step gives X_1 = -X_0 with
    I - A X_1 = 4 I, so the refinement stops and hands back X_0 unchanged."""
    p = 300
    A = wl.matern32(wl.uniform_points(np.random.default_rng(4), p, 2), 0.1, 1.0, 1e-2)
    inv = np.linalg.inv(A)
    X0 = 3.0 * 0.5 * (inv + inv.T)
    dA, dX = torch.from_numpy(A).cuda(), torch.from_numpy(X0.copy()).cuda()
    prec = ibmi.IBMI_MIXED if precision == "mixed" else ibmi.IBMI_FP64
    s, res = ibmi.ibmi_refine(dA, dX, precision=prec, tol=1e-11, ns_max=6)
    assert s == ibmi.IBMI_NOT_CONVERGED and res["ns_steps"] == 1, res
    assert np.array_equal(dX.cpu().numpy(), X0)
    assert res["resid_f"] == pytest.approx(O.residual_f(A, X0), rel=1e-9)


def test_bounded_wait_expires_cleanly(ibmi):
    s = ibmi.ibmi_selftest_wait_timeout()
    assert s == ibmi.IBMI_ERR_TIMEOUT, ibmi.ibmi_status_string(s)
    torch.cuda.synchronize()
    # the context is still usable: a mixed inversion right after succeeds
    A = wl.matern32(wl.uniform_points(np.random.default_rng(6), 256, 2), 0.1, 1.0, 1e-2)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(256, K=2, h=16, tol=1e-10, precision=ibmi.IBMI_MIXED, ns_theta=0.5)
    s2, res = ibmi.ibmi_invert(plan, dA, dH)
    plan.close()
    assert s2 == ibmi.IBMI_OK and O.residual_f(A, dH.cpu().numpy()) <= 1e-10, res


def test_reported_flops_follow_the_cost_model(ibmi):
    p, K, h, r = 384, 3, 16, 4
    A = wl.matern32(wl.uniform_points(np.random.default_rng(9), p, 2), 0.1, 1.0, 1e-2)
    sets = O.partition(p, K, h)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(p, K=K, h=h, tol=0.0, max_sweeps=r)
    s, res = ibmi.ibmi_invert(plan, dA, dH)
    plan.close()
    want = O.plan_flops(p, sets) + r * (O.sweep_flops(p, sets) + 2.0 * p ** 3)
    assert s == ibmi.IBMI_NOT_CONVERGED and res["flops"] == pytest.approx(want, rel=1e-12)
