"""Partition and ordering search (ibmi_tune) and the device permutation.

A Matern-3/2 matrix on points in random order is the case Section 5.7 warns
about: contiguous sets over an order that scatters near points converge
slowly or not at all.  The search over orderings from the points' coordinates
must pick one that keeps near points together, and the inverse computed with
its choice, permuted back, must be A's inverse.
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


def test_permute_is_symmetric_indexing_of_the_lower_triangle(ibmi):
    rng = np.random.default_rng(0)
    p = 300
    S = rng.standard_normal((p, p))
    S = S + S.T
    perm = rng.permutation(p)
    An = S.copy()
    An[np.triu_indices(p, 1)] = np.nan      # only the lower triangle may be read
    dA = torch.from_numpy(An).cuda()
    dB = torch.empty_like(dA)
    ibmi.ibmi_permute(dA, perm, dB)
    B = dB.cpu().numpy()
    np.testing.assert_array_equal(B, S[np.ix_(perm, perm)])
    dC = torch.empty_like(dA)
    ibmi.ibmi_permute(dB, perm, dC, inverse=True)
    np.testing.assert_array_equal(dC.cpu().numpy(), S)


def test_tune_picks_a_local_ordering_and_its_inverse_is_correct(ibmi):
    p = 1024
    rng = np.random.default_rng(5)
    pts = wl.uniform_points(rng, p, 2, sort=False)          # random order
    A = wl.matern32(pts, 0.1, 1.0, 1e-2)
    orders = [ibmi.IBMI_ORDER_XSORT, ibmi.IBMI_ORDER_HILBERT, ibmi.IBMI_ORDER_KD, ibmi.IBMI_ORDER_REDBLACK]
    perms = [ibmi.ibmi_order_points(pts, o) for o in orders]
    dA = torch.from_numpy(A).cuda()
    s, best, cands = ibmi.ibmi_tune(dA, perms, precision=ibmi.IBMI_MIXED, tol=1e-10, max_sweeps=60,
                                    ns_theta=0.9)
    assert s == ibmi.IBMI_OK, best
    assert best["order"] in (0, 1, 2), best              # x-sort, Hilbert or k-d
    by_order = {}
    for c in cands:
        by_order.setdefault(c["order"], []).append(c)
    ok = {o: [c for c in cs if c["status"] == 0] for o, cs in by_order.items()}
    fastest = {o: min((c["seconds"] for c in cs), default=float("inf")) for o, cs in ok.items()}
    print({o: (len(ok[o]), len(by_order[o]), round(fastest[o] * 1e3, 2)) for o in sorted(by_order)})
    assert fastest[0] < fastest[-1] and fastest[0] < fastest[3]   # sorted beats random and red-black
    # the inverse with the chosen ordering and partition, permuted back
    q = perms[best["order"]]
    dAp = torch.empty_like(dA)
    ibmi.ibmi_permute(dA, q, dAp)
    plan = ibmi.ibmi_plan(p, K=best["K"], h=best["h"], precision=ibmi.IBMI_MIXED, tol=1e-10, max_sweeps=60,
                          ns_theta=0.9)
    dHp = torch.empty_like(dA)
    st, res = ibmi.ibmi_invert(plan, dAp, dHp)
    plan.close()
    assert st == ibmi.IBMI_OK and res["sweeps"] == best["sweeps"], (res, best)
    dH = torch.empty_like(dA)
    ibmi.ibmi_permute(dHp, q, dH, inverse=True)
    H = dH.cpu().numpy()
    assert O.residual_f(A, H) <= 1e-10
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-8 * np.abs(inv).max()
