"""Partial (block-diagonal) inverse on the GPU, ibmi_invert_block_diag, vs
the oracle's two-set recurrence (Section 6 Discussion).

Fixed-sweep blocks agree to 1e-12 in relative Frobenius norm (both sides
FP64; only summation orders differ) and equal the diagonal blocks of the
GPU's own full iterate to the same tolerance; converged blocks reach the stop
quantity and match LAPACK's inverse blocks.
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


def matern(p, seed):
    return wl.matern32(wl.uniform_points(np.random.default_rng(seed), p, 2), 0.1, 1.0, 1e-2)


def run_bd(ibmi, A, h, D0=None, **kw):
    p = A.shape[0]
    sets = O.partition(p, 2, h)
    (l1, h1), (l2, h2) = sets
    m1, m2 = h1 - l1, h2 - l2
    dA = torch.from_numpy(A).cuda()
    D = torch.zeros(m1 * m1 + m2 * m2, dtype=torch.float64, device="cuda")
    if D0 is not None:
        D[m1 * m1:] = torch.from_numpy(np.ascontiguousarray(D0).ravel()).cuda()
    plan = ibmi.ibmi_plan(p, K=2, h=h, **kw)
    s, res = ibmi.ibmi_invert_block_diag(plan, dA, D)
    torch.cuda.synchronize()
    plan.close()
    Dh = D.cpu().numpy()
    return s, res, Dh[:m1 * m1].reshape(m1, m1), Dh[m1 * m1:].reshape(m2, m2), sets


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("p,h", [(300, 0), (333, 20), (640, 64)])
@pytest.mark.parametrize("r", [1, 3])
def test_fixed_sweeps_match_the_oracle_and_the_full_iterate(ibmi, p, h, r):
    A = matern(p, 61)
    s, res, D1, D2, sets = run_bd(ibmi, A, h, tol=0.0, max_sweeps=r)
    assert s == ibmi.IBMI_NOT_CONVERGED and res["sweeps"] == r, res
    ref = O.ibmi_block_diagonal(A, sets, tol=0.0, max_sweeps=r)
    assert rel(D1, ref.d1) <= 1e-12 and rel(D2, ref.d2) <= 1e-12
    assert res["resid_f"] == pytest.approx(ref.resid_rows, rel=1e-9)
    # the same blocks as the full GPU iterate
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(p, K=2, h=h, tol=0.0, max_sweeps=r)
    ibmi.ibmi_invert(plan, dA, dH)
    plan.close()
    H = dH.cpu().numpy()
    (l1, h1), (l2, h2) = sets
    assert rel(D1, H[:h1, :h1]) <= 1e-12 and rel(D2, H[l2:, l2:]) <= 1e-12


@pytest.mark.parametrize("p,h", [(512, 0), (1024, 64)])
def test_converged_blocks(ibmi, p, h):
    A = matern(p, 62)
    s, res, D1, D2, sets = run_bd(ibmi, A, h, tol=1e-10, max_sweeps=500)
    ref = O.ibmi_block_diagonal(A, sets, tol=1e-10, max_sweeps=500)
    assert s == ibmi.IBMI_OK and ref.status == "converged", res
    assert res["resid_f"] <= 1e-10
    assert abs(res["sweeps"] - ref.sweeps) <= 1
    inv = np.linalg.inv(A)
    (l1, h1), (l2, h2) = sets
    sc = np.abs(inv).max()
    assert np.abs(D1 - inv[:h1, :h1]).max() <= 1e-8 * sc
    assert np.abs(D2 - inv[l2:, l2:]).max() <= 1e-8 * sc
    print(f"p={p} h={h}: {res['sweeps']} sweeps (oracle {ref.sweeps}), rows residual {res['resid_f']:.2e}")


def test_user_and_complement_inverse_guesses(ibmi):
    p, h = 400, 24
    A = matern(p, 63)
    sets = O.partition(p, 2, h)
    (l1, h1), (l2, h2) = sets
    rng = np.random.default_rng(3)
    G = rng.standard_normal((h2 - l2, h2 - l2))
    T0 = np.eye(h2 - l2) + 0.05 * (G + G.T)
    s, res, D1, D2, _ = run_bd(ibmi, A, h, D0=T0, tol=0.0, max_sweeps=2, init=ibmi.IBMI_INIT_USER)
    ref = O.ibmi_block_diagonal(A, sets, tol=0.0, max_sweeps=2, t0=T0)
    assert rel(D1, ref.d1) <= 1e-12 and rel(D2, ref.d2) <= 1e-12
    h0 = O.schur_initial_guess(A, sets)
    s, res, D1, D2, _ = run_bd(ibmi, A, h, tol=0.0, max_sweeps=2, init=ibmi.IBMI_INIT_SCHUR)
    ref = O.ibmi_block_diagonal(A, sets, tol=0.0, max_sweeps=2, t0=h0[l2:, l2:])
    assert rel(D1, ref.d1) <= 1e-12 and rel(D2, ref.d2) <= 1e-12


def test_rejects_plans_it_cannot_serve(ibmi):
    A = torch.from_numpy(matern(256, 64)).cuda()
    D = torch.zeros(256 * 256, dtype=torch.float64, device="cuda")
    for kw in (dict(K=3, h=8), dict(K=2, h=8, precision=ibmi.IBMI_MIXED)):
        plan = ibmi.ibmi_plan(256, **kw)
        s, _ = ibmi.ibmi_invert_block_diag(plan, A, D)
        plan.close()
        assert s == ibmi.IBMI_ERR_INVALID_ARG
