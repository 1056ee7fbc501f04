"""Only the lower triangle of A is read: with NaN in the strict upper triangle
every entry point returns the bits it returns for the full symmetric A."""
import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibmi():
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as m
    return m


def _pair(p, seed=5):
    rng = np.random.default_rng(seed)
    A = wl.matern32(wl.uniform_points(rng, p, 2), 0.1, 1.0, 1e-2)
    B = A.copy()
    B[np.triu_indices(p, 1)] = np.nan
    return A, B


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_invert_reads_lower_triangle_only(ibmi, precision):
    p = 333
    A, B = _pair(p)
    prec = ibmi.IBMI_MIXED if precision == "mixed" else ibmi.IBMI_FP64
    outs = []
    for M in (A, B):
        dA = torch.from_numpy(M).cuda()
        dH = torch.empty_like(dA)
        plan = ibmi.ibmi_plan(p, K=3, h=7, precision=prec, tol=1e-10, max_sweeps=200,
                              ns_theta=0.5 if prec == ibmi.IBMI_MIXED else 0.0)
        s, r = ibmi.ibmi_invert(plan, dA, dH)
        torch.cuda.synchronize()
        plan.close()
        outs.append((s, r["sweeps"], r["ns_steps"], dH.cpu().numpy()))
    assert outs[0][:3] == outs[1][:3]
    assert np.array_equal(outs[0][3], outs[1][3])
    assert np.isfinite(outs[1][3]).all()


def test_residuals_and_refine_read_lower_triangle_only(ibmi):
    p = 300
    A, B = _pair(p, seed=6)
    H = np.linalg.inv(A) * (1 + 1e-6)
    H = (H + H.T) / 2
    dH = torch.from_numpy(H).cuda()
    vals = []
    for M in (A, B):
        dA = torch.from_numpy(M).cuda()
        r64 = ibmi.ibmi_residual(dA, dH)
        rtc = ibmi.ibmi_residual_tc(dA, dH)
        X = dH.clone()
        s, res = ibmi.ibmi_refine(dA, X, precision=ibmi.IBMI_MIXED, tol=1e-12, ns_max=4)
        vals.append((r64, rtc, s, res["ns_steps"], X.cpu().numpy()))
    assert vals[0][:4] == vals[1][:4]
    assert np.array_equal(vals[0][4], vals[1][4])


def test_batched_reads_lower_triangle_only(ibmi):
    pairs = [_pair(p, seed=10 + p) for p in (96, 200)]
    outs = []
    for k in (0, 1):
        As = [torch.from_numpy(pr[k]).cuda() for pr in pairs]
        Hs = [torch.empty_like(a) for a in As]
        s, res = ibmi.ibmi_invert_batched(As, Hs, workers=2, autotune=0)
        torch.cuda.synchronize()
        outs.append((s, [r["sweeps"] for r in res], [h.cpu().numpy() for h in Hs]))
    assert outs[0][:2] == outs[1][:2]
    for a, b in zip(outs[0][2], outs[1][2]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_padded_leading_dimensions(ibmi, precision):
    """A and H stored with row pitches above p give the bits of contiguous
    storage (padding untouched in H, ignored in A)."""
    p, lda, ldh = 301, 301 + 37, 301 + 5
    A, _ = _pair(p, seed=9)
    prec = ibmi.IBMI_MIXED if precision == "mixed" else ibmi.IBMI_FP64
    kw = dict(K=3, h=9, precision=prec, tol=1e-10, max_sweeps=200, ns_theta=0.9 if prec == ibmi.IBMI_MIXED else 0.0)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(p, **kw)
    s0, r0 = ibmi.ibmi_invert(plan, dA, dH)
    Apad = torch.full((p, lda), float("nan"), dtype=torch.float64, device="cuda")
    Apad[:, :p] = dA
    Hpad = torch.full((p, ldh), -7.0, dtype=torch.float64, device="cuda")
    s1, r1 = ibmi.ibmi_invert(plan, Apad[:, :p], Hpad[:, :p])
    torch.cuda.synchronize()
    plan.close()
    assert (s0, r0["sweeps"], r0["ns_steps"]) == (s1, r1["sweeps"], r1["ns_steps"])
    assert np.array_equal(dH.cpu().numpy(), Hpad[:, :p].cpu().numpy())
    assert torch.all(Hpad[:, p:] == -7.0)
