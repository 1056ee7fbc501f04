"""Host logic of the Newton-Schulz tail plan (csrc/tail_plan.h), compiled on
the CPU with g++: pair counts, step counts and bounds against their closed
forms, the group choice against its definition, and the digit groups the plan
takes on trajectories measured on GB300 (C2 and a squared-exponential p = 2048
matrix), so that a change of the plan's arithmetic shows here."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_06377_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstring>
#include "tail_plan.h"
using namespace ibmi::tail;
int main() {
  char c[8];
  while (std::scanf("%7s", c) == 1) {
    if (!std::strcmp(c, "P")) { int q, a, b; std::scanf("%d %d %d", &q, &a, &b); std::printf("%d\n", pairs(q, a, b)); }
    else if (!std::strcmp(c, "S")) { double r, t; std::scanf("%lf %lf", &r, &t); std::printf("%d\n", steps(r, t)); }
    else if (!std::strcmp(c, "B")) { int k; double t; std::scanf("%d %lf", &k, &t); std::printf("%.17g\n", bound(k, t)); }
    else if (!std::strcmp(c, "T")) { double r, t; std::scanf("%lf %lf", &r, &t); std::printf("%.17g\n", target(r, t)); }
    else if (!std::strcmp(c, "RF")) { int q, qc; double g, a; std::scanf("%d %lf %d %lf", &q, &g, &qc, &a);
      std::printf("%.17g\n", residual_floor(q, g, qc, a)); }
    else if (!std::strcmp(c, "UF")) { int q; double r, a; std::scanf("%d %lf %lf", &q, &r, &a);
      std::printf("%.17g\n", update_floor(q, r, a)); }
    else if (!std::strcmp(c, "RG")) { double t, g, a; int qc, lo, hi; std::scanf("%lf %lf %d %lf %d %d", &t, &g, &qc, &a, &lo, &hi);
      std::printf("%d\n", residual_groups(t, g, qc, a, lo, hi)); }
    else if (!std::strcmp(c, "UG")) { double r, a, t; int qf; std::scanf("%lf %lf %lf %d", &r, &a, &t, &qf);
      std::printf("%d\n", update_groups(r, a, t, qf)); }
    else if (!std::strcmp(c, "CG")) { double r, t; int qm; std::scanf("%lf %lf %d", &r, &t, &qm);
      std::printf("%d\n", correction_groups(r, t, qm)); }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("tail_plan")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def call(*lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.split()
        return [float(x) if ("." in x or "e" in x or "n" in x.lower()) else int(x) for x in out]
    return call


def test_pair_counts(plan):
    # s < 10 digits of X, u < 8 of A: all (q+1)(q+2)/2 pairs up to q = 7, then 8 per group
    got = plan(*[f"P {q} 10 8" for q in range(10)])
    assert got == [(q + 1) * (q + 2) // 2 for q in range(8)] + [44, 52]
    assert plan("P 4 5 5", "P 3 5 5") == [15, 10]


def test_steps_count_squarings(plan):
    tol = 1e-10
    for rho in (0.5, 0.19, 7.75e-3, 1.3e-4, 2.2e-7, 1e-9, 1e-12):
        n, r = 0, rho
        while r > 0.25 * tol and n < 12:
            r, n = r * r, n + 1
        assert plan(f"S {rho!r} {tol!r}") == [max(n, 1)]
    assert plan("S 2.0 1e-10") == [12]


def test_bound_reaches_tolerance(plan):
    tol = 1e-10
    assert plan(f"B 0 {tol!r}")[0] == 0.25 * tol
    prev = 0.0
    for k in range(1, 6):
        b = plan(f"B {k} {tol!r}")[0]
        assert b > prev
        prev = b
        r = b
        for _ in range(k):   # k steps that multiply rho^2 by 16 end at tol / 4
            r = 16.0 * r * r
        assert r <= 0.25 * tol * (1 + 1e-12)
    # target: half the bound for the steps after this one
    assert plan(f"T 7.75e-3 {tol!r}")[0] == pytest.approx(0.5 * plan(f"B 2 {tol!r}")[0], rel=1e-15)


def test_residual_groups_is_the_fewest_within_target(plan):
    g, qc, amp = 7.8732e-06, 5, 672.5
    for t in (1e-2, 1.4e-4, 6.25e-7, 1e-9, 1.25e-11, 1e-16):
        q = plan(f"RG {t!r} {g!r} {qc} {amp!r} 4 9")[0]
        floors = plan(*[f"RF {x} {g!r} {qc} {amp!r}" for x in range(4, 9)])
        fits = [x for x, f in zip(range(4, 9), floors) if f <= t]
        assert q == (fits[0] if fits else 9)
    # each group is 2^-7 of the one before
    f5, f6 = plan(f"RF 5 {g!r} {qc} {amp!r}", f"RF 6 {g!r} {qc} {amp!r}")
    assert f5 / f6 == pytest.approx(128.0, rel=1e-15)
    # nothing measured (exact digits) takes the fewest; an unusable measure takes all
    assert plan("RG 1e-12 0 5 672.5 4 9", "RG 1e-12 nan 5 672.5 4 9", "RG 1e-12 inf 5 672.5 4 9") == [4, 9, 9]


def test_plan_on_measured_c2_trajectory(plan):
    """C2 (p = 4096 Matern-3/2, K = 8, h = 32, theta 0.9) measured on GB300:
    rho and the norm g of the last kept group at each tail residual; the plan
    keeps 5, 6, 9, 9 groups and updates with 3, 3, 4 (10, 10, 15 pairs)."""
    tol, amp = 1e-10, 672.5
    rho0, g5 = 7.7506e-03, 7.8732e-06
    assert plan(f"RG {plan(f'T {rho0!r} {tol!r}')[0]!r} {g5!r} 5 {amp!r} 4 9") == [5]   # 5 is enough: no extension
    assert plan(f"UG {rho0!r} {amp!r} {tol!r} 4") == [3]
    fl0 = plan(f"RF 5 {g5!r} 5 {amp!r}")[0] + plan(f"UF 3 {rho0!r} {amp!r}")[0]
    rho_hat1 = max(rho0 * rho0, fl0)
    assert plan(f"RG {plan(f'T {rho_hat1!r} {tol!r}')[0]!r} {g5!r} 5 {amp!r} 4 9") == [6]
    rho1, g6 = 1.3175e-04, 5.9504e-08
    assert plan(f"RG {plan(f'T {rho1!r} {tol!r}')[0]!r} {g6!r} 6 {amp!r} 4 9")[0] <= 6
    assert plan(f"UG {rho1!r} {amp!r} {tol!r} 4") == [3]
    fl1 = plan(f"RF 6 {g6!r} 6 {amp!r}")[0] + plan(f"UF 3 {rho1!r} {amp!r}")[0]
    rho_hat2 = max(rho1 * rho1, fl1)
    assert plan(f"RG {plan(f'T {rho_hat2!r} {tol!r}')[0]!r} {g6!r} 6 {amp!r} 4 9") == [9]
    rho2, g9 = 2.1996e-07, 5.4128e-14
    assert plan(f"UG {rho2!r} {amp!r} {tol!r} 4") == [4]
    fl2 = plan(f"RF 9 {g9!r} 9 {amp!r}")[0] + plan(f"UF 4 {rho2!r} {amp!r}")[0]
    assert max(rho2 * rho2, fl2) <= tol   # the next residual is expected to certify: all groups


def test_plan_extends_the_first_residual_of_a_harder_matrix(plan):
    """Squared-exponential p = 2048 (3-D points, length scale 0.2, nugget
    1e-3), measured: amp = 6964; the first residual's 5 groups are not enough
    for its step and are extended to 6, and the update keeps all 15 pairs
    (10 cost this matrix a fifth step in the probe)."""
    tol, amp, rho0, g5 = 1e-10, 6964.0, 1.9184e-01, 7.3075e-05
    t = plan(f"T {rho0!r} {tol!r}")[0]
    assert plan(f"RG {t!r} {g5!r} 5 {amp!r} 4 9") == [6]
    assert plan(f"UG {rho0!r} {amp!r} {tol!r} 4") == [4]
    rho2 = 1.7829e-04   # third residual: still 15 pairs
    assert plan(f"UG {rho2!r} {amp!r} {tol!r} 4") == [4]


# ------------------------------------------------------------------------
# The error model against an exact emulation of the digit-sliced products
# (CPU, p = 128): row-scaled 7-bit digits of X and A as integers, the group
# sums as exact int64 products, one symmetrised Newton-Schulz step in FP64.

def _digits(X, nd):
    """F = rint(x 2^(55-e)) with |x| < 2^e per row; digit s (rounded, 7 bits
    apart) weighs 2^(e - 6 - 7 s)."""
    import numpy as np
    p = X.shape[0]
    mx = np.max(np.abs(X), axis=1)
    e = np.array([math.frexp(float(v))[1] if v > 0 else 0 for v in mx], dtype=np.int64)
    D = np.zeros((nd, p, p), dtype=np.int64)
    for i in range(p):
        for j in range(p):
            f = int(round(math.ldexp(float(X[i, j]), 55 - int(e[i]))))
            for s in range(nd):
                sh = 49 - 7 * s
                d = (f + (1 << (sh - 1))) >> sh
                f -= d << sh
                D[s, i, j] = d
    return D, e


def _product(DX, ex, DB, eb, q):
    """sum over pairs s + u <= q of digit products of X B^T, and group q's part."""
    import numpy as np
    p = DX.shape[1]
    C = np.zeros((p, p))
    last = None
    for g in range(q + 1):
        Tg = np.zeros((p, p), dtype=np.int64)
        for s in range(g + 1):
            if s < DX.shape[0] and g - s < DB.shape[0]:
                Tg += DX[s] @ DB[g - s].T
        last = Tg.astype(float) * 2.0 ** (-7 * g)
        C += last
    scale = np.ldexp(1.0, (ex[:, None] + eb[None, :] - 12).astype(np.int64))
    return C * scale, last * scale


def _cases():
    import numpy as np
    import workloads as wl
    yield "se", wl.squared_exp(wl.uniform_points(np.random.default_rng(7), 128, 3), 0.3, nugget=1e-3)
    yield "matern", wl.matern32(wl.uniform_points(np.random.default_rng(8), 128, 2), 0.1, nugget=1e-2)
    yield "kms", wl.kms(128, 0.9)


def _iterate(A, eps):
    import numpy as np
    p = A.shape[0]
    P = np.random.default_rng(1).standard_normal((p, p))
    P = 0.5 * (P + P.T)
    X = np.linalg.inv(A) @ (np.eye(p) - eps * P / np.linalg.norm(P, 2))
    return 0.5 * (X + X.T)


def test_residual_floor_model_against_emulation(plan):
    """The floor a truncated residual leaves after one symmetrised step is
    what residual_floor predicts (which carries a factor 2 of margin): the
    model stays within [1, 3] times the emulated floor for the groups the plan
    uses (q >= 3), with amp from 30 to 1500."""
    import numpy as np
    for name, A in _cases():
        p = A.shape[0]
        X = _iterate(A, 1e-3)
        amp = np.linalg.norm(A) * np.linalg.norm(X) / p
        DX, ex = _digits(X, 7)
        DA, ea = _digits(A, 7)

        def step(Q):
            Xn = X + X @ Q.T
            return np.eye(p) - A @ (0.5 * (Xn + Xn.T))
        E_exact = step(np.eye(p) - X @ A)
        for q in (3, 4, 5):
            C, last = _product(DX, ex, DA, ea, q)
            g = np.linalg.norm(last) / math.sqrt(p)
            floor = np.linalg.norm(step(np.eye(p) - C) - E_exact) / math.sqrt(p)
            model = plan(f"RF {q} {float(g)!r} {q} {float(amp)!r}")[0]
            assert floor <= model <= 3.0 * floor, (name, q, floor, model)


def test_update_floor_model_is_conservative_at_small_order(plan):
    """The update's constant was measured at orders 2048-4096 (c = 75..260,
    kUpdateFloor 512); the row-scaled digits' error grows with the order, and
    at p = 128 the emulated floor sits below the model."""
    import numpy as np
    for name, A in _cases():
        p = A.shape[0]
        for eps in (1e-2, 1e-4):
            X = _iterate(A, eps)
            amp = np.linalg.norm(A) * np.linalg.norm(X) / p
            Q = np.eye(p) - X @ A
            rho = np.linalg.norm(Q) / math.sqrt(p)
            DX, ex = _digits(X, 5)
            DQ, eq = _digits(Q, 5)
            E_exact = np.eye(p) - A @ (X + X @ Q.T)
            for qu in (3, 4):
                U, _ = _product(DX, ex, DQ, eq, qu)
                floor = np.linalg.norm(np.eye(p) - A @ (X + 0.5 * (U + U.T)) - E_exact) / math.sqrt(p)
                assert floor <= plan(f"UF {qu} {float(rho)!r} {float(amp)!r}")[0], (name, eps, qu)


def test_correction_groups(plan):
    """The batched tail's correction groups: the fewest (at least 5) with
    rho 2^(-7(q+1)) 3e6 <= 1e-2 tol, from the definition, and never more
    than the cap."""
    def ref(r, t, qm):
        q = 5
        while q < qm and r * 2.0 ** (-7 * (q + 1)) * 3e6 > 1e-2 * t:
            q += 1
        return q
    cases = [(1e-9, 1e-10), (1e-6, 1e-10), (1.1e-6, 1e-10), (1e-4, 1e-10), (3e-4, 1e-10), (1e-2, 1e-10),
             (1e-6, 1e-12), (0.5, 1e-14), (1e-8, 1e-6)]
    got = plan(*[f"CG {r} {t} 9" for r, t in cases])
    assert got == [ref(r, t, 9) for r, t in cases]
    assert got[1] == 5 and got[3] == 6 and got[7] == 9   # 21 pairs up to rho = 1e-6 at tol 1e-10; capped
    assert plan("CG 1e-2 1e-10 6") == [6]
