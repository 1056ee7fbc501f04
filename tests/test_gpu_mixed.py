"""Mixed-precision GPU path (tcgen05 BF16x3 sweep products) vs the FP64 oracle.

Fixed-sweep trajectories are held to the error of a CPU model of the mixed
arithmetic (``bf16x3_sweeps`` below): the iterate kept as an FP32 master,
each operand of a sweep product cut into two BF16 slices (hi = bf16(x),
lo = bf16(x - hi)), the three slice products hi*hi + hi*lo + lo*hi summed in
FP32, H[I, I] = A_I^{-1} - P rounded to FP32.  That model carries every
rounding of the GPU path except the order of the FP32 accumulations (and W's
34-bit digit formation, far below them); the accumulation order changes each
sum by about sqrt(n) 2^-24 of its terms, the same order as the model's own
accumulation error, so the GPU's distance to the FP64 oracle is bounded by
twice the model's.  Converged runs must reach ||I - A H||_F / sqrt(p) <= 1e-10
after the Newton-Schulz tail, like the oracle.
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


def run(ibmi, A, **kw):
    p = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    dH = torch.empty_like(dA)
    plan = ibmi.ibmi_plan(p, precision=ibmi.IBMI_MIXED, **kw)
    s, res = ibmi.ibmi_invert(plan, dA, dH)
    torch.cuda.synchronize()
    plan.close()
    return s, res, dH.cpu().numpy()


def matern(p, seed):
    rng = np.random.default_rng(seed)
    return wl.matern32(wl.uniform_points(rng, p, 2), 0.1, 1.0, 1e-2)


def _bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even) on the bit patterns."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16).astype(np.uint32)).view(np.float32)


def _x3(a, b):
    """a @ b from two BF16 slices of each FP32 operand, three slice products,
    FP32 accumulation."""
    a = np.asarray(a, np.float32)
    b = np.asarray(b, np.float32)
    a0, b0 = _bf16(a), _bf16(b)
    a1, b1 = _bf16(a - a0), _bf16(b - b0)
    return (a0 @ b0 + a0 @ b1 + a1 @ b0).astype(np.float32)


def bf16x3_sweeps(A, sets, r):
    """r sweeps of eq. IBMI in the mixed arithmetic (model, see the module
    docstring), with the FP64 invariants of the oracle."""
    p = A.shape[0]
    invs = [O.block_invariants(A, lo, hi) for lo, hi in sets]
    H = np.eye(p, dtype=np.float32)
    for _ in range(r):
        for inv in invs:
            I, ic = np.arange(inv.lo, inv.hi), inv.ic
            X = -_x3(inv.w, H[np.ix_(ic, ic)])
            P = _x3(X, inv.w.T)
            P = np.tril(P) + np.tril(P, -1).T          # lower tiles, mirrored
            H[np.ix_(I, ic)] = X
            H[np.ix_(ic, I)] = X.T
            H[np.ix_(I, I)] = (inv.ainv - P.astype(np.float64)).astype(np.float32)
    return H.astype(np.float64)


@pytest.mark.parametrize("p,K,h", [(256, 2, 0), (333, 4, 7), (517, 5, 16), (640, 3, 64)])
@pytest.mark.parametrize("r", [1, 3])
def test_mixed_fixed_sweeps_close_to_oracle(ibmi, p, K, h, r):
    A = matern(p, 21)
    sets = O.partition(p, K, h)
    ref = O.ibmi(A, sets, tol=0.0, max_sweeps=r)
    s, res, H = run(ibmi, A, K=K, h=h, tol=0.0, max_sweeps=r)
    assert s == ibmi.IBMI_NOT_CONVERGED and res["sweeps"] == r
    nrm = np.linalg.norm(ref.h)
    err = np.linalg.norm(H - ref.h) / nrm
    model = np.linalg.norm(bf16x3_sweeps(A, sets, r) - ref.h) / nrm
    print(f"p={p} K={K} h={h} r={r} rel err {err:.2e} (BF16x3 model {model:.2e})")
    assert err <= 2.0 * model
    assert np.array_equal(H, H.T)


def test_mixed_kms_one_sweep(ibmi):
    A = wl.c1_kms()
    s, res, H = run(ibmi, A, K=2, h=0, tol=1e-10, ns_theta=0.5)
    assert s == ibmi.IBMI_OK
    ref = O.spd_inverse(A)
    assert np.abs(H - ref).max() < 1e-9


@pytest.mark.parametrize("p,K,h", [(512, 4, 16), (700, 3, 40)])
def test_mixed_converged_with_newton_schulz(ibmi, p, K, h):
    A = matern(p, 22)
    ref = O.ibmi(A, O.partition(p, K, h), tol=1e-10, max_sweeps=300, ns_theta=0.5)
    s, res, H = run(ibmi, A, K=K, h=h, tol=1e-10, max_sweeps=300, ns_theta=0.5)
    assert ref.status == "converged" and s == ibmi.IBMI_OK, res
    assert O.residual_f(A, H) <= 1e-10
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-8 * np.abs(inv).max()
    print("mixed", res["sweeps"], res["ns_steps"], "oracle", ref.sweeps, ref.ns_steps)


def test_mixed_full_size_c2(ibmi):
    A = wl.c2_matern()
    p = A.shape[0]
    s, res, H = run(ibmi, A, K=8, h=32, tol=1e-10, max_sweeps=200, ns_theta=0.5)
    assert s == ibmi.IBMI_OK and res["resid_f"] <= 1e-10, res
    rng = np.random.default_rng(1)
    rows = rng.choice(p, 16, replace=False)
    R = np.eye(p)[rows] - A[rows] @ H
    assert np.abs(R).max() < 1e-9
    print("c2 mixed", res)


@pytest.mark.parametrize("p", [200, 1000, 4160])
def test_tc_residual_matches_fp64(ibmi, p):
    """The sliced error-free tensor-core residual agrees with FP64 evaluations
    at the level of FP64 rounding, both far from and at the inverse."""
    A = matern(p, 31)
    rng = np.random.default_rng(2)
    inv = np.linalg.inv(A)
    inv = 0.5 * (inv + inv.T)
    for H in (inv, inv + 1e-6 * (lambda g: g + g.T)(rng.standard_normal((p, p)))):
        dA, dH = torch.from_numpy(A).cuda(), torch.from_numpy(np.ascontiguousarray(H)).cuda()
        got = ibmi.ibmi_residual_tc(dA, dH)
        want = O.residual_f(A, H)
        dfma = ibmi.ibmi_residual(dA, dH)
        print(f"p={p} tc={got:.6e} oracle={want:.6e} dfma={dfma:.6e}")
        assert abs(got - want) <= 1e-3 * want + 1e-14
        assert abs(got - dfma) <= 1e-3 * dfma + 1e-14


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("p", [300, 1024])
def test_refine_newton_schulz_entry(ibmi, precision, p):
    """eq. newton on its own: from a perturbed inverse (||I - A X_0|| < 1) the
    tail converges quadratically to the FP64 floor; the residual it reports is
    the oracle's."""
    A = matern(p, 41)
    inv = np.linalg.inv(A)
    rng = np.random.default_rng(5)
    N = rng.standard_normal((p, p))
    X0 = 0.5 * (inv + inv.T) + 1e-6 * (N + N.T)
    dA, dX = torch.from_numpy(A).cuda(), torch.from_numpy(X0).cuda()
    prec = ibmi.IBMI_MIXED if precision == "mixed" else ibmi.IBMI_FP64
    s, res = ibmi.ibmi_refine(dA, dX, precision=prec, tol=1e-11, ns_max=6)
    X = dX.cpu().numpy()
    assert s == ibmi.IBMI_OK and 1 <= res["ns_steps"] <= 3, res
    assert O.residual_f(A, X) <= 1e-11
    assert res["resid_f"] == pytest.approx(O.residual_f(A, X), rel=0.05, abs=1e-13)
    assert np.array_equal(X, X.T)


def test_refine_rejects_bad_args(ibmi):
    A = torch.eye(8, dtype=torch.float64, device="cuda")
    s, _ = ibmi.ibmi_refine(A, A.clone(), precision=5)
    assert s == ibmi.IBMI_ERR_INVALID_ARG


def test_mixed_full_size_c3_random_spd(ibmi):
    """p = 8192 random SPD (Q diag(lambda) Q^T, lambda log-uniform in [1, 1e4]),
    two sets with 2048-row overlap: the BF16x3 sweep stalls, escalates to three
    slices, and the Newton-Schulz tail reaches the tolerance.  Checked on
    sampled rows of the residual and sampled columns of the inverse."""
    A = wl.c3_random_spd()
    p = A.shape[0]
    s, res, H = run(ibmi, A, K=2, h=1024, tol=1e-10, max_sweeps=500, ns_theta=0.5)
    assert s == ibmi.IBMI_OK and res["resid_f"] <= 1e-10, res
    rng = np.random.default_rng(3)
    rows = rng.choice(p, 8, replace=False)
    R = np.eye(p)[rows] - A[rows] @ H
    assert np.abs(R).max() < 1e-9
    cols = rng.choice(p, 2, replace=False)
    X = np.linalg.solve(A, np.eye(p)[:, cols])
    assert np.abs(H[:, cols] - X).max() <= 1e-8 * np.abs(X).max()
    print("c3 mixed", res)


@pytest.mark.parametrize("ell", [0.3, 0.5])
def test_mixed_floor_hands_over_by_radius(ibmi, ell):
    """A squared-exponential matrix on 3-D points (kappa 2e5 to 4e5) with two
    large blocks: the sweeps reach their mixed-precision floor with
    ||I - A H||_F above 8 theta, yet the spectral radius of I - X A is far below
    1, so the Newton-Schulz tail of eq. newton converges from there."""
    rng = np.random.default_rng(7)
    A = wl.squared_exp(wl.uniform_points(rng, 960, 3), ell, 1.0, 1e-3)
    s, res, H = run(ibmi, A, K=2, h=48, tol=1e-10, ns_theta=0.5, max_sweeps=300)
    print(res)
    assert s == ibmi.IBMI_OK and res["ns_steps"] >= 1
    assert O.residual_f(A, H) <= 1e-10
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-6 * np.abs(inv).max()


def test_mixed_not_spd_reported_like_oracle(ibmi):
    p = 200
    A = wl.random_spd(p, 6, 1.0, 1e2)
    A[150, 150] = -5.0
    s, res, _ = run(ibmi, A, K=2, h=10, tol=1e-10, ns_theta=0.5)
    ref = O.ibmi(A, O.partition(p, 2, 10), tol=1e-10)
    assert s == ibmi.IBMI_ERR_NOT_SPD and ref.status == "not_spd"
    assert res["bad_block"] == ref.bad_block and res["bad_pivot"] == ref.bad_pivot


@pytest.mark.parametrize("pivot", [300, 1900])
def test_mixed_not_spd_large_blocks_reported_like_oracle(ibmi, pivot):
    """Blocks of order >= 1024 factorise with tensor-core updates: a negative
    pivot is still found, in the first block column (300) or after several
    tensor-core updates (1900 in the second block), at the oracle's block and
    pivot."""
    p, K, h = 2400, 2, 16
    A = wl.random_spd(p, 66, 1.0, 1e2)
    A[pivot, pivot] = -5.0
    s, res, _ = run(ibmi, A, K=K, h=h, tol=1e-10, ns_theta=0.9)
    sets = O.partition(p, K, h)
    ref = O.ibmi(A, sets, tol=1e-10, max_sweeps=1)
    assert s == ibmi.IBMI_ERR_NOT_SPD and ref.status == "not_spd"
    assert res["bad_block"] == ref.bad_block and res["bad_pivot"] == ref.bad_pivot, (res, ref.bad_block, ref.bad_pivot)


def test_mixed_nonfinite_reported(ibmi):
    """A NaN outside every diagonal block reaches H through W and the sweeps
    and is reported as IBMI_ERR_NONFINITE (never as a converged result)."""
    p = 256
    A = matern(p, 31)
    A[250, 3] = A[3, 250] = np.nan        # sets [0, 128) and [128, 256): off-block
    s, res, _ = run(ibmi, A, K=2, h=0, tol=1e-10, ns_theta=0.5)
    assert s == ibmi.IBMI_ERR_NONFINITE


def test_sliced_residual_propagates_nonfinite(ibmi):
    """An Inf or NaN in H (or A) makes the FP64-accurate sliced residual NaN
    instead of a finite value from meaningless digits."""
    p = 200
    A = matern(p, 33)
    H = np.linalg.inv(A)
    for bad in (np.nan, np.inf):
        Hb = H.copy()
        Hb[17, 5] = Hb[5, 17] = bad
        v = ibmi.ibmi_residual_tc(torch.from_numpy(A).cuda(), torch.from_numpy(Hb).cuda())
        assert not np.isfinite(v)
    v = ibmi.ibmi_residual_tc(torch.from_numpy(A).cuda(), torch.from_numpy(H).cuda())
    assert np.isfinite(v) and v < 1e-12


def test_mixed_single_set_is_direct_inverse(ibmi):
    """One set covering the matrix: the block inverse is the answer, for a
    mixed-precision plan as for an FP64 one."""
    p = 160
    A = matern(p, 35)
    s, res, H = run(ibmi, A, K=1, tol=1e-12)
    assert s == ibmi.IBMI_OK and res["sweeps"] == 1
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-12 * np.abs(inv).max()


def test_mixed_large_blocks_tensor_core_block_inverse(ibmi):
    """Blocks of order >= 1024 take A_I^{-1} = Y^T Y from the sliced tensor-core
    product: the converged inverse is the FP64 one, and fixed-sweep iterates
    follow the oracle's as closely as with the FP64 block inverse."""
    p, K, h = 2300, 2, 50
    A = matern(p, 37)
    s, res, H = run(ibmi, A, K=K, h=h, tol=1e-10, ns_theta=0.9, max_sweeps=300)
    assert s == ibmi.IBMI_OK
    rf = O.residual_f(A, H)
    # the reported value (a tail from order 2048 certifies by a correction of
    # the last full residual) is the FP64 residual of the returned H
    assert rf <= 1e-10 and res["resid_f"] == pytest.approx(rf, rel=1e-3, abs=1e-14), (rf, res)
    inv = np.linalg.inv(A)
    assert np.abs(H - inv).max() <= 1e-7 * np.abs(inv).max()
    ref = O.ibmi(A, O.partition(p, K, h), tol=0.0, max_sweeps=2)
    s, res, H = run(ibmi, A, K=K, h=h, tol=0.0, max_sweeps=2)
    assert np.linalg.norm(H - ref.h) / np.linalg.norm(ref.h) < 5e-4


def test_mixed_large_blocks_factorise_on_tensor_cores(ibmi):
    """Blocks of order >= 1024 take the Cholesky's trailing updates beyond each
    256-column block column as exact digit products on the tensor cores
    (FP64-accurate): fixed-sweep iterates follow the oracle's (FP64
    factorisation) as closely as the FP64-factorised path does, and the
    converged inverse certifies 1e-10 against the oracle's residual."""
    p, K, h = 4200, 2, 0
    A = wl.random_spd(p, 61, 1.0, 1e3)
    ref = O.ibmi(A, O.partition(p, K, h), tol=0.0, max_sweeps=2)
    s, res, H = run(ibmi, A, K=K, h=h, tol=0.0, max_sweeps=2)
    err = np.linalg.norm(H - ref.h) / np.linalg.norm(ref.h)
    print(f"p {p}: 2-sweep iterate vs oracle, relative Frobenius {err:.3e}")
    assert err < 5e-4
    assert np.array_equal(H, H.T)   # blocks of 2100 rows: the a4 finish runs in the product's epilogue
    s, res, H = run(ibmi, A, K=K, h=h, tol=1e-10, ns_theta=0.9, max_sweeps=300)
    assert s == ibmi.IBMI_OK, res
    rf = O.residual_f(A, H)
    assert rf <= 1e-10 and res["resid_f"] == pytest.approx(rf, rel=1e-3, abs=1e-14), (rf, res)


def test_bench_configuration_c2_matches_the_oracle(ibmi):
    """The exact configuration the benchmark times (p = 4096 Matern-3/2,
    K = 8, h = 32, theta = 0.9, tol 1e-10), element by element against the
    oracle's own converged solve of the same input.

    Bound: H_gpu - H_ora = A^{-1} ((I - A H_ora) - (I - A H_gpu)), so
    ||H_gpu - H_ora||_F <= ||A^{-1}||_2 (||R_gpu||_F + ||R_ora||_F), and
    ||A^{-1}||_2 <= 1 / nugget = 100 because the Matern-3/2 kernel matrix is
    positive semidefinite and the workload adds 1e-2 I."""
    A = wl.c2_matern()
    p = A.shape[0]
    s, res, H = run(ibmi, A, K=8, h=32, tol=1e-10, max_sweeps=500, ns_theta=0.9, ns_max=8, check_every=1)
    assert s == ibmi.IBMI_OK, res
    rf = O.residual_f(A, H)
    assert rf <= 1e-10 and res["resid_f"] == pytest.approx(rf, rel=1e-3, abs=1e-14), (rf, res)
    ref = O.ibmi(A, O.partition(p, 8, 32), tol=1e-10, max_sweeps=500, ns_theta=0.9)
    assert ref.status == "converged"
    bound = 100.0 * (rf + ref.resid_f) * np.sqrt(p)
    d = H - ref.h
    err_f, err_max = np.linalg.norm(d), np.abs(d).max()
    print(f"c2 bench config: gpu {res['sweeps']} sweeps + {res['ns_steps']} NS, rho_F {rf:.3e}; oracle "
          f"{ref.sweeps} + {ref.ns_steps}, rho_F {ref.resid_f:.3e}; ||H-H_ora||_F {err_f:.3e} "
          f"(rel {err_f / np.linalg.norm(ref.h):.3e}), max-abs {err_max:.3e}, bound {bound:.3e}")
    assert err_f <= bound and err_max <= bound
    assert np.array_equal(H, H.T)
