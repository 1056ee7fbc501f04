"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests re-types an oracle formula: each compares the oracle with a
closed form, an exact brute force, a library routine, an identity of the
method's analysis (Lemma / Theorem of Section 3) or a value printed in the paper.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as wl
from oracle import ibmi_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def rand_spd(p, seed, cond=50.0):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    lam = np.exp(rng.uniform(0.0, math.log(cond), p))
    a = (q * lam) @ q.T
    return 0.5 * (a + a.T)


def kms_inverse(p, rho):
    """Textbook tridiagonal inverse of the AR(1) matrix rho^|i-j|."""
    inv = np.zeros((p, p))
    c = 1.0 / (1.0 - rho * rho)
    for i in range(p):
        inv[i, i] = c * (1.0 + rho * rho) if 0 < i < p - 1 else c
        if i + 1 < p:
            inv[i, i + 1] = inv[i + 1, i] = -rho * c
    return inv


# ------------------------------------------------------------- partition --

def test_partition_layout_c2():
    # Section 4: end sets m + h, interior sets m + 2h; p = 4096, K = 8, h = 32.
    sets = O.partition(4096, 8, 32)
    assert sets[0] == (0, 544) and sets[-1] == (3552, 4096)
    assert [hi - lo for lo, hi in sets] == [544] + [576] * 6 + [544]
    for (l0, h0), (l1, h1) in zip(sets, sets[1:]):
        assert h0 - l1 == 64          # consecutive overlap 2h
    assert O.partition(256, 2, 0) == [(0, 128), (128, 256)]


def test_partition_uneven_covers():
    for p, K, h in [(320, 3, 16), (1000, 7, 5), (65, 4, 3)]:
        sets = O.partition(p, K, h)
        cov = np.zeros(p, int)
        for lo, hi in sets:
            cov[lo:hi] += 1
        assert cov.min() >= 1 and sets[0][0] == 0 and sets[-1][1] == p


# ------------------------------------------------------ direct inverse ----

def _exact_inverse(a_frac):
    n = len(a_frac)
    m = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(a_frac)]
    for c in range(n):
        piv = next(r for r in range(c, n) if m[r][c] != 0)
        m[c], m[piv] = m[piv], m[c]
        inv = 1 / m[c][c]
        m[c] = [v * inv for v in m[c]]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c]
                m[r] = [vr - f * vc for vr, vc in zip(m[r], m[c])]
    return [[float(v) for v in row[n:]] for row in m]


@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_spd_inverse_vs_exact_rational(p):
    rng = np.random.default_rng(p)
    g = rng.integers(-4, 5, size=(p, p))
    a_int = g @ g.T + p * np.eye(p, dtype=int)          # integer SPD
    exact = np.array(_exact_inverse([[Fraction(int(v)) for v in row] for row in a_int]))
    got = O.spd_inverse(a_int.astype(np.float64))
    assert np.max(np.abs(got - exact)) <= 1e-13 * np.max(np.abs(exact))


def test_cholesky_vs_lapack():
    a = rand_spd(60, 1)
    np.testing.assert_allclose(O.cholesky(a), np.linalg.cholesky(a), rtol=0, atol=1e-12)


def test_spd_inverse_kms_closed_form():
    a = wl.kms(256, 0.5)
    np.testing.assert_allclose(O.spd_inverse(a), kms_inverse(256, 0.5), rtol=0, atol=1e-13)


def test_spd_inverse_sherman_morrison():
    p, a, b = 50, 0.7, 0.4
    want = (np.eye(p) - b / (a + p * b) * np.ones((p, p))) / a
    np.testing.assert_allclose(O.spd_inverse(wl.compound_symmetry(p, a, b)), want, rtol=0, atol=1e-13)


def test_not_spd_detected():
    a = rand_spd(40, 2)
    a[25, 25] = -1.0
    res = O.ibmi(a, O.partition(40, 2, 4), 1e-10)
    assert res.status == "not_spd" and res.bad_block == 1


# ------------------------------------------------- block update (eq. IBMI) --

@pytest.mark.parametrize("lo,hi", [(0, 13), (9, 27), (30, 40), (0, 40 - 1)])
def test_exact_schur_complement_gives_exact_inverse(lo, hi):
    """eq. BMIQ: with T equal to the exact inverse Schur complement
    (A^{-1})[I^c, I^c], one application of eq. IBMI returns A^{-1}."""
    a = rand_spd(40, 3)
    ainv = np.linalg.inv(a)
    ainv = 0.5 * (ainv + ainv.T)
    h = ainv.copy()
    h[lo:hi, :] = 7.0          # garbage in the rows/cols being rewritten
    h[:, lo:hi] = -3.0
    O.block_update(h, O.block_invariants(a, lo, hi))
    np.testing.assert_allclose(h, ainv, rtol=0, atol=1e-11 * np.abs(ainv).max())
    assert np.array_equal(h, h.T)


def test_c1_kms_converges_in_one_sweep():
    a = wl.c1_kms()
    res = O.ibmi(a, O.partition(256, 2, 0), tol=1e-12)
    assert res.status == "converged" and res.sweeps == 1
    np.testing.assert_allclose(res.h, kms_inverse(256, 0.5), rtol=0, atol=5e-15)


@pytest.mark.parametrize("p,rho,c", [(16, 0.5, 2.0), (256, 0.5, 2.0), (40, 0.8, 3.0)])
def test_kms_trajectory_closed_form(p, rho, c):
    """Two blocks, T_0 = c I.  Lemma of Section 3 with A_1^{-1} A_12 = rho e_m v^T
    gives the error after r sweeps exactly:
    delta rho^{4r-2} [[1, -rho], [-rho, rho^2]] on rows/cols (m-1, m), zero
    elsewhere, delta = (c (1 - rho^p) - 1) / (1 - rho^2)."""
    a = wl.kms(p, rho)
    m = p // 2
    sig = kms_inverse(p, rho)
    delta = (c * (1.0 - rho ** p) - 1.0) / (1.0 - rho * rho)
    for r in (1, 2, 3):
        res = O.ibmi(a, [(0, m), (m, p)], tol=0.0, max_sweeps=r, h0=c * np.eye(p))
        want = sig.copy()
        e = delta * rho ** (4 * r - 2)
        want[m - 1, m - 1] += e
        want[m - 1, m] -= e * rho
        want[m, m - 1] -= e * rho
        want[m, m] += e * rho * rho
        assert res.sweeps == r
        np.testing.assert_allclose(res.h, want, rtol=0, atol=2e-14 * max(1.0, abs(delta)))
        # paper's estimate (eq. error) on I_2: rank one, closed form
        est = abs(delta) * rho ** (4 * r - 1) * math.sqrt((1 - rho * rho) * (1 - rho ** p))
        assert O.paper_error(a, res.h, m, p) == pytest.approx(est, rel=1e-9, abs=1e-15)


def test_compound_symmetry_trajectory_closed_form():
    """aI + b11^T, two halves of size m: M = lam (11^T/m), lam = (mb/(a+mb))^2,
    so by the Lemma the error of H[I_2, I_2] after r sweeps is
    lam^{2r} [1 - 1/a + b m / (a (a + p b))] 11^T / m for T_0 = I."""
    p, a_, b_ = 64, 0.5, 1.0
    m = p // 2
    A = wl.compound_symmetry(p, a_, b_)
    sig = (np.eye(p) - b_ / (a_ + p * b_) * np.ones((p, p))) / a_
    lam = (m * b_ / (a_ + m * b_)) ** 2
    c0 = 1.0 - 1.0 / a_ + b_ * m / (a_ * (a_ + p * b_))
    P = np.ones((m, m)) / m
    for r in (1, 2, 5):
        res = O.ibmi(A, [(0, m), (m, p)], tol=0.0, max_sweeps=r)
        err = res.h[m:, m:] - sig[m:, m:]
        np.testing.assert_allclose(err, lam ** (2 * r) * c0 * P, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed,p,m", [(5, 24, 10), (6, 40, 23), (7, 48, 24)])
def test_lemma_recurrence_and_theorem_bound(seed, p, m):
    """Lemma (Section 3): E_r = M^r E_0 (M^T)^r with M = A_2^{-1} A_21 A_1^{-1} A_12;
    Theorem: ||E_r||_2 <= ||M||_2^{2r} ||E_0||_2; and rho(M) < 1."""
    a = rand_spd(p, seed)
    rng = np.random.default_rng(seed + 100)
    g = rng.standard_normal((p - m, p - m))
    t0 = g @ g.T / (p - m) + np.eye(p - m)                     # SPD initial guess
    h0 = np.eye(p)
    h0[m:, m:] = t0
    A1, A2, A12 = a[:m, :m], a[m:, m:], a[:m, m:]
    M = np.linalg.solve(A2, A12.T) @ np.linalg.solve(A1, A12)
    sig2 = np.linalg.inv(a)[m:, m:]
    E0 = t0 - sig2
    assert max(abs(np.linalg.eigvals(M))) < 1.0
    nM = np.linalg.norm(M, 2)
    for r in (1, 2, 4):
        res = O.ibmi(a, [(0, m), (m, p)], tol=0.0, max_sweeps=r, h0=h0)
        Er = res.h[m:, m:] - sig2
        Mr = np.linalg.matrix_power(M, r)
        want = Mr @ E0 @ Mr.T
        np.testing.assert_allclose(Er, want, rtol=0, atol=1e-10 * max(1.0, np.abs(E0).max()))
        assert np.linalg.norm(Er, 2) <= nM ** (2 * r) * np.linalg.norm(E0, 2) * (1 + 1e-9) + 1e-13


def test_symmetry_exact():
    a = rand_spd(70, 8)
    res = O.ibmi(a, O.partition(70, 3, 5), tol=0.0, max_sweeps=3)
    assert np.array_equal(res.h, res.h.T)


@pytest.mark.parametrize("p,rho,K,h", [(64, 0.5, 4, 2), (96, 0.8, 3, 1), (120, 0.9, 5, 4), (64, 0.8, 8, 2),
                                       (50, 0.95, 2, 1)])
def test_kms_overlapping_sets_exact_in_one_sweep(p, rho, K, h):
    """AR(1)/KMS, several overlapping sets swept left to right (Algorithm 1).
    For a set I = [lo, hi) the coupling to the columns left of it is rank one,
    A[i, j] = rho^(i-lo) rho^(lo-j), and rho^(i-lo) is the first column of A_I,
    so A_I^{-1} maps it to the first unit vector; on the right it is the last
    column.  Hence W = A_I^{-1} A_{I,I^c} is zero except in its first and
    last rows, and eq. IBMI leaves every row of H[I, :] but the last one
    depending on T only through its left part, which the tridiagonal inverse
    (whose A_{I'}^{-1} block of the previous set differs from A^{-1} only in
    that set's last row and column) makes exact.  With overlap the next set
    rewrites that last row, and the last set has no right complement: one
    sweep gives A^{-1} from any symmetric starting H."""
    a = wl.kms(p, rho)
    sig = kms_inverse(p, rho)
    sets = O.partition(p, K, h)
    g = np.random.default_rng(p).standard_normal((p, p))
    for h0 in (3.0 * np.eye(p), g + g.T):
        res = O.ibmi(a, sets, tol=0.0, max_sweeps=1, h0=h0)
        assert res.sweeps == 1
        np.testing.assert_allclose(res.h, sig, rtol=0, atol=5e-15 * np.max(np.abs(sig)) * p)


@pytest.mark.parametrize("K", [3, 4, 6])
def test_kms_nonoverlapping_sets_contract_by_rho4(K):
    """The same matrix without overlap: each boundary between consecutive sets
    keeps an error that the next sweep multiplies by rho^4, the rate of the
    two-block trajectory above (rho^(4r-2)); once the boundaries' errors have
    settled the ratio of consecutive sweeps' errors is rho^4."""
    p, rho = 60, 0.8
    a = wl.kms(p, rho)
    sig = kms_inverse(p, rho)
    sets = O.partition(p, K, 0)
    errs = [np.max(np.abs(O.ibmi(a, sets, tol=0.0, max_sweeps=r, h0=2.0 * np.eye(p)).h - sig))
            for r in range(4, 8)]
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 / e0 == pytest.approx(rho ** 4, rel=1e-6)


def test_multiblock_overlap_converges_to_inverse():
    """Remark of Section 3: the multi-block overlapping sweep converges in
    practice; checked against LAPACK's inverse."""
    a = wl.c2_matern(p=512, seed=11)
    res = O.ibmi(a, O.partition(512, 4, 16), tol=1e-11, max_sweeps=300)
    assert res.status == "converged"
    inv = np.linalg.inv(a)
    assert np.max(np.abs(res.h - inv)) <= 1e-8 * np.max(np.abs(inv))


# ----------------------------------------------------------- residuals ----

def test_residual_closed_forms():
    p = 64
    a = wl.kms(p, 0.6)
    assert O.residual_f(a, kms_inverse(p, 0.6)) < 1e-15
    assert O.residual_f(a, np.zeros((p, p))) == pytest.approx(1.0, abs=1e-15)
    h = kms_inverse(p, 0.6)
    i, j, eps = 5, 40, 1e-3
    h[i, j] += eps
    # I - A (A^{-1} + eps e_i e_j^T) = -eps (A e_i) e_j^T
    want = eps * np.linalg.norm(a[:, i]) / math.sqrt(p)
    assert O.residual_f(a, h) == pytest.approx(want, rel=1e-9)


def test_paper_error_zero_at_inverse():
    a = rand_spd(30, 9)
    assert O.paper_error(a, np.linalg.inv(a), 10, 20) < 1e-12


def test_newton_schulz_squares_the_residual():
    """eq. newton: I - A X_{n+1} = (I - A X_n)^2."""
    a = rand_spd(50, 10)
    x = np.linalg.inv(a) + 1e-3 * rand_spd(50, 11) / 50
    R0 = np.eye(50) - a @ x
    x1, nr = O.newton_schulz_step(a, x)
    assert nr == pytest.approx(np.linalg.norm(R0), rel=1e-12)
    np.testing.assert_allclose(np.eye(50) - a @ x1, R0 @ R0, rtol=0, atol=1e-12)


def test_hybrid_tail_reaches_tolerance():
    a = wl.random_spd(192, seed=12, lam_lo=1.0, lam_hi=1e3)
    res = O.ibmi(a, O.partition(192, 2, 48), tol=1e-12, max_sweeps=200, ns_theta=0.5)
    assert res.status == "converged" and res.ns_steps >= 1
    inv = np.linalg.inv(a)
    assert np.max(np.abs(res.h - inv)) <= 1e-9 * np.max(np.abs(inv))


# ------------------------------------------------------ paper's numbers ----

def test_table2_exp_1d_one_iteration():
    g = json.load(open(os.path.join(HERE, "golden", "table2_1d_exp.json")))
    for row in g["rows"]:
        p = row["p"]
        a = wl.exp_1d(p)
        h = int(round(0.2 * (p // 2) / 2))      # 20% overlap of the core width
        res = O.ibmi(a, O.partition(p, 2, h), tol=g["tol"], stop_rule="paper", max_sweeps=50)
        assert res.status == "converged" and res.sweeps == row["iterations"]
        err = np.linalg.norm(res.h - np.linalg.inv(a), 2)
        assert err <= 10 * row["error_2norm"]


# ------------------------------------------------------------ flop counts ----

class _CountingArray(np.ndarray):
    """ndarray whose matrix products add their multiply-add count
    (rows x inner x columns) to a shared tally and return plain arrays."""
    tally = [0]

    @staticmethod
    def _count(a, b):
        a, b = np.asarray(a), np.asarray(b)
        inner = a.shape[-1]
        rows = a.shape[0] if a.ndim == 2 else 1
        cols = b.shape[1] if b.ndim == 2 else 1
        _CountingArray.tally[0] += rows * inner * cols
        return a @ b

    def __matmul__(self, other):
        return self._count(self, other)

    def __rmatmul__(self, other):
        return self._count(other, self)


def _textbook_chol_inverse_fmas(m):
    """Multiply-adds of the column Cholesky (one length-j dot per entry of
    column j on and below the diagonal) and of the two triangular solves with
    m right-hand sides (a length-i dot per row i and right-hand side), counted
    by walking the loops."""
    n = 0
    for j in range(m):
        for _ in range(j, m):
            n += j
    for i in range(m):
        n += 2 * i * m
    return n


def test_flop_counts_match_counted_operations():
    """plan_flops / sweep_flops (Section 4 cost model, FMA = 2 flops) against
    the multiply-adds the oracle's own products perform (counted on the
    operands) plus loop counts of the textbook factorisation and solves."""
    p, K, h = 224, 3, 6
    a = wl.matern32(wl.uniform_points(np.random.default_rng(3), p, 2), 0.2, 1.0, 1e-2)
    sets = O.partition(p, K, h)
    ac = a.view(_CountingArray)
    for lo, hi in sets:
        m = hi - lo
        _CountingArray.tally[0] = 0
        inv = O.block_invariants(ac, lo, hi)            # counts the W product
        counted = 2 * (_CountingArray.tally[0] + _textbook_chol_inverse_fmas(m))
        want = O.plan_flops(p, [(lo, hi)])
        assert abs(want - counted) <= 2.0 / m * counted, (m, want, counted)
        _CountingArray.tally[0] = 0
        h_it = np.eye(p).view(_CountingArray)
        inv.w = inv.w.view(_CountingArray)
        O.block_update(h_it, inv)                        # W T and X W^T
        assert O.sweep_flops(p, [(lo, hi)]) == 2 * _CountingArray.tally[0]
    assert O.sweep_flops(p, sets) == sum(O.sweep_flops(p, [s]) for s in sets)


# ------------------------------------------------------ stop-test cadence ----

def test_check_every_tests_less_often_on_the_same_iterates():
    """Algorithm 1 with the stop test every 3rd sweep: the iterates are those
    of the per-sweep test (the test does not touch H), the tests fall on
    sweeps 3, 6, ... and the last one, and convergence is seen at the first
    tested sweep at or after the per-sweep run's stopping sweep."""
    a = wl.matern32(wl.uniform_points(np.random.default_rng(8), 160, 2), 0.1, 1.0, 1e-2)
    sets = O.partition(160, 4, 4)
    every = O.ibmi(a, sets, tol=0.0, max_sweeps=7)
    third = O.ibmi(a, sets, tol=0.0, max_sweeps=7, check_every=3)
    assert np.array_equal(every.h, third.h)
    assert [r for r, _, _ in third.history] == [3, 6, 7]
    rf = {r: v for r, v, _ in every.history}
    for r, v, _ in third.history:
        assert v == rf[r]
    ref = O.ibmi(a, sets, tol=1e-6, max_sweeps=200)
    assert ref.status == "converged" and ref.sweeps % 3 != 0
    got = O.ibmi(a, sets, tol=1e-6, max_sweeps=200, check_every=3)
    r_star = 3 * math.ceil(ref.sweeps / 3)
    assert got.status == "converged" and got.sweeps == r_star
    assert np.array_equal(got.h, O.ibmi(a, sets, tol=0.0, max_sweeps=r_star).h)


# ----------------------------------------------- Newton-Schulz divergence ----

def test_newton_schulz_divergence_keeps_the_previous_iterate():
    """eq. newton converges only when the spectral radius of I - A X is below
    1.  KMS with the initial guess 100 I leaves, after one two-block sweep, an
    error of q rho^2 [[1, -rho], [-rho, rho^2]] with q ~ 520 (the KMS
    trajectory above), far outside that region: the step grows the residual,
    so the tail stops and returns the iterate of the hand-over with its
    residual."""
    p, rho = 16, 0.9
    a = wl.kms(p, rho)
    sets = O.partition(p, 2, 0)
    h0 = 100.0 * np.eye(p)
    one = O.ibmi(a, sets, tol=0.0, max_sweeps=1, h0=h0)
    assert max(abs(np.linalg.eigvals(np.eye(p) - a @ one.h))) > 1.0
    res = O.ibmi(a, sets, tol=1e-12, max_sweeps=50, ns_theta=1e9, h0=h0)
    assert res.status == "ns_diverged" and res.sweeps == 1 and res.ns_steps == 1
    assert np.array_equal(res.h, one.h)
    assert res.resid_f == one.resid_f
    assert res.history[-1][2] > res.resid_f      # the rejected step's residual


# ------------------------------------------------ initial guess (Table 6) ----

def test_schur_initial_guess_kms_closed_form():
    """For KMS the complement block of the first set is again a KMS matrix,
    whose inverse is the tridiagonal closed form."""
    p, rho = 48, 0.7
    a = wl.kms(p, rho)
    sets = O.partition(p, 3, 2)
    h0 = O.schur_initial_guess(a, sets)
    hi1 = sets[0][1]
    np.testing.assert_allclose(h0[hi1:, hi1:], kms_inverse(p - hi1, rho), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(h0[:hi1], np.eye(p)[:hi1])
    np.testing.assert_array_equal(h0[:, :hi1], np.eye(p)[:, :hi1])


def test_schur_initial_guess_two_blocks_is_the_second_block_inverse():
    """Two non-overlapping sets: I_1^c = I_2, so T_0 = A_2^{-1} (LAPACK)."""
    a = rand_spd(40, 21)
    sets = O.partition(40, 2, 0)
    h0 = O.schur_initial_guess(a, sets)
    np.testing.assert_allclose(h0[20:, 20:], np.linalg.inv(a[20:, 20:]), rtol=0, atol=1e-10)


# ------------------------------------- partial (block-diagonal) inverse ----

@pytest.mark.parametrize("p,h", [(40, 0), (48, 5), (60, 12)])
@pytest.mark.parametrize("r", [1, 2, 5])
def test_block_diagonal_equals_the_full_iterates_blocks(p, h, r):
    """The two-set recurrence on the diagonal blocks alone reproduces, sweep
    by sweep, the diagonal blocks of the full Algorithm 1 iterate, and its
    stop quantity is the norm of the full residual's rows I_2."""
    a = rand_spd(p, 30 + p)
    sets = O.partition(p, 2, h)
    (l1, h1), (l2, h2) = sets
    full = O.ibmi(a, sets, tol=0.0, max_sweeps=r)
    part = O.ibmi_block_diagonal(a, sets, tol=0.0, max_sweeps=r)
    assert part.sweeps == r
    np.testing.assert_allclose(part.d1, full.h[:h1, :h1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(part.d2, full.h[l2:, l2:], rtol=0, atol=1e-13)
    R = full.h[l2:] @ a - np.eye(p)[l2:]
    assert part.resid_rows == pytest.approx(np.linalg.norm(R) / math.sqrt(p), rel=1e-10)


def test_block_diagonal_kms_closed_form_and_convergence():
    """KMS, two non-overlapping sets, identity guess: converged blocks are
    those of the tridiagonal closed-form inverse; a random SPD matrix with
    overlapping sets converges to LAPACK's blocks."""
    p = 64
    a = wl.kms(p, 0.6)
    res = O.ibmi_block_diagonal(a, O.partition(p, 2, 0), tol=1e-13)
    inv = kms_inverse(p, 0.6)
    assert res.status == "converged"
    np.testing.assert_allclose(res.d1, inv[:32, :32], rtol=0, atol=1e-12)
    np.testing.assert_allclose(res.d2, inv[32:, 32:], rtol=0, atol=1e-12)
    b = rand_spd(50, 77, cond=20.0)
    sets = O.partition(50, 2, 6)
    res = O.ibmi_block_diagonal(b, sets, tol=1e-13, max_sweeps=400)
    invb = np.linalg.inv(b)
    assert res.status == "converged"
    np.testing.assert_allclose(res.d1, invb[:31, :31], rtol=0, atol=1e-10)
    np.testing.assert_allclose(res.d2, invb[19:, 19:], rtol=0, atol=1e-10)
