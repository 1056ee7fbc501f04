"""Initial guess T_0 = A_{I_1^c}^{-1} (IBMI_INIT_SCHUR, Section 5.6, Table 6)
on the GPU against the oracle run from the same initial iterate.

FP64 fixed-sweep trajectories agree to 1e-12 in relative Frobenius norm (both
sides FP64, only summation orders differ); mixed runs must converge to
||I - A H||_F / sqrt(p) <= 1e-10 like the oracle, for a complement block
below order 1024 (FP64 Y^T Y) and one above it (sliced Y^T Y on the tensor
cores).
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


def run(ibmi, A, **kw):
    p = A.shape[0]
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(p, init=ibmi.IBMI_INIT_SCHUR, **kw)
    s, res = ibmi.ibmi_invert(plan, dA, dH)
    torch.cuda.synchronize()
    plan.close()
    return s, res, dH.cpu().numpy()


@pytest.mark.parametrize("p,K,h", [(333, 4, 7), (640, 2, 64)])
@pytest.mark.parametrize("r", [1, 2])
def test_fp64_fixed_sweeps_from_the_complement_inverse(ibmi, p, K, h, r):
    A = matern(p, 51)
    sets = O.partition(p, K, h)
    ref = O.ibmi(A, sets, tol=0.0, max_sweeps=r, h0=O.schur_initial_guess(A, sets))
    s, res, H = run(ibmi, A, K=K, h=h, tol=0.0, max_sweeps=r)
    assert s == ibmi.IBMI_NOT_CONVERGED and res["sweeps"] == r
    assert np.linalg.norm(H - ref.h) <= 1e-12 * np.linalg.norm(ref.h)


@pytest.mark.parametrize("p,K,h", [(1536, 2, 128), (2560, 2, 128)])
def test_mixed_converges_from_the_complement_inverse(ibmi, p, K, h):
    A = matern(p, 52)
    sets = O.partition(p, K, h)
    s, res, H = run(ibmi, A, K=K, h=h, tol=1e-10, max_sweeps=300, precision=ibmi.IBMI_MIXED, ns_theta=0.9)
    assert s == ibmi.IBMI_OK, res
    assert O.residual_f(A, H) <= 1e-10
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-8 * np.abs(inv).max()
    ref = O.ibmi(A, sets, tol=1e-10, max_sweeps=300, ns_theta=0.9, h0=O.schur_initial_guess(A, sets))
    print(f"p={p}: gpu {res['sweeps']} sweeps + {res['ns_steps']} NS; oracle {ref.sweeps} + {ref.ns_steps}")
    assert ref.status == "converged"


def test_complement_block_not_spd_is_reported(ibmi):
    """K = 3 sets whose own diagonal blocks are SPD, while the complement block
    of the first set is not: rows of set 2 only and of set 3 only never meet
    inside a set, so a large coupling between them shows only there."""
    p, K, h = 96, 3, 2
    A = np.eye(p)
    sets = O.partition(p, K, h)
    (l1, h1), (l2, h2), (l3, h3) = sets
    i, j = h1 + 1, h3 - 2          # i in set 2 only, j in set 3 only
    assert l2 <= i < l3 and h2 <= j
    A[i, j] = A[j, i] = 3.0
    for lo, hi in sets:
        np.linalg.cholesky(A[lo:hi, lo:hi])          # each set's block is SPD
    with pytest.raises(O.NotSPD):
        O.spd_inverse(A[h1:, h1:])
    s, res, _ = run(ibmi, A, K=K, h=h, tol=1e-10)
    assert s == ibmi.IBMI_ERR_NOT_SPD and res["bad_block"] == K, res
