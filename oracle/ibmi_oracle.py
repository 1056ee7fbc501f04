"""Plain FP64 reference implementation of IBMI (Iterative Block Matrix Inversion).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the CPU
baseline leg of bench.py, never by the product path.  It shares no code with
the CUDA kernels; the only thing both sides read is the seeded input generator
module ``workloads``.

Every routine follows the paper's statement of the step it implements, in the
paper's order and notation, with numpy's matrix product as the only library
primitive.  Nothing is blocked, fused or reordered.

Notation: A is the SPD matrix (the paper's Q), H the current approximation of
A^{-1}, I = [lo, hi) a contiguous index set and Ic its complement
[0, lo) U [hi, p).  T = H[Ic, Ic] is the approximation of the inverse Schur
complement used by the approximate block inversion formula (eq. IBMI).

Readings taken where the paper is silent (each is listed in the design notes):
  * index sets: core width m = p/K, end sets widened by h on one side and
    interior sets by h on both sides (Section 4 cost model: |I_1| = |I_K| = m+h,
    |I_k| = m+2h otherwise), boundaries b_k = floor(k p / K);
  * the (I, I) block is symmetrised, (S + S^T)/2, and H[Ic, I] is written as the
    transpose of the same X that is written to H[I, Ic];
  * the stopping quantity defaults to ||I - A H||_F / sqrt(p); the paper's
    estimate (eq. error) is evaluated on the last set I_K and is available as
    an alternative stop rule;
  * the Newton-Schulz tail (eq. newton) is entered once the unscaled
    ||I - A H||_F falls below theta and is symmetrised each step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "NotSPD", "partition", "complement", "cholesky", "forward_subst", "backward_subst",
    "spd_inverse", "block_invariants", "block_update", "residual_f", "paper_error",
    "newton_schulz_step", "ibmi", "IbmiResult", "sweep_flops", "plan_flops", "schur_initial_guess",
    "ibmi_block_diagonal", "BlockDiagResult",
]


class NotSPD(Exception):
    """Cholesky met a non-positive pivot: the block is not positive definite."""

    def __init__(self, pivot: int, block: int = -1):
        super().__init__(f"non-positive pivot {pivot} in block {block}")
        self.pivot = pivot
        self.block = block


# ----------------------------------------------------------------- sets ----

def partition(p: int, K: int, h: int) -> list[tuple[int, int]]:
    """Contiguous, overlapping index sets I_1..I_K (Section 2.3, multi-block
    overlapping case; sizes as in the Section 4 cost model).

    Core k covers [b_k, b_{k+1}) with b_k = floor(k p / K); each set extends
    its core by h on every side that has a neighbour, so consecutive sets
    overlap by 2h.  h = 0 gives the non-overlapping partition.
    """
    if K < 1 or p < K or h < 0:
        raise ValueError("need 1 <= K <= p and h >= 0")
    b = [(k * p) // K for k in range(K + 1)]
    return [(max(0, b[k] - h), min(p, b[k + 1] + h)) for k in range(K)]


def complement(p: int, lo: int, hi: int) -> np.ndarray:
    """I^c = {0..p-1} minus [lo, hi), in increasing order."""
    return np.concatenate([np.arange(0, lo), np.arange(hi, p)])


# ------------------------------------------------- direct SPD inversion ----

def cholesky(a: np.ndarray) -> np.ndarray:
    """Lower-triangular L with A = L L^T (the Cholesky factorisation used for
    the diagonal blocks, Section 1 and Section 4).  Column-by-column
    (left-looking) definition."""
    n = a.shape[0]
    L = np.zeros((n, n))
    for j in range(n):
        d = a[j, j] - L[j, :j] @ L[j, :j]
        if not d > 0.0:
            raise NotSPD(j)
        L[j, j] = math.sqrt(d)
        L[j + 1:, j] = (a[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    return L


def forward_subst(L: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve L Z = B for lower-triangular L, one row at a time."""
    n = L.shape[0]
    Z = np.zeros_like(B, dtype=np.float64)
    for i in range(n):
        Z[i] = (B[i] - L[i, :i] @ Z[:i]) / L[i, i]
    return Z


def backward_subst(U: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Solve U X = B for upper-triangular U, one row at a time from the bottom."""
    n = U.shape[0]
    X = np.zeros_like(B, dtype=np.float64)
    for i in range(n - 1, -1, -1):
        X[i] = (B[i] - U[i, i + 1:] @ X[i + 1:]) / U[i, i]
    return X


def spd_inverse(a: np.ndarray) -> np.ndarray:
    """A^{-1} through the Cholesky factor (Section 1): A = L L^T, then solve
    L z_i = e_i and L^T h_i = z_i for all unit vectors e_i at once."""
    L = cholesky(a)
    Z = forward_subst(L, np.eye(a.shape[0]))
    return backward_subst(L.T, Z)


# --------------------------------------------------------- block update ----

@dataclass
class BlockInv:
    lo: int
    hi: int
    ic: np.ndarray      # I^c indices
    ainv: np.ndarray    # A_I^{-1}                      (m x m)
    w: np.ndarray       # A_I^{-1} A_{I, I^c}            (m x n)


def block_invariants(a: np.ndarray, lo: int, hi: int) -> BlockInv:
    """The parts of eq. IBMI that do not depend on the iterate: A_I^{-1} and
    A_I^{-1} A_{I,I^c} (the product the cost analysis of Section 4 counts four
    times per set)."""
    p = a.shape[0]
    ic = complement(p, lo, hi)
    ainv = spd_inverse(a[lo:hi, lo:hi])
    w = ainv @ a[lo:hi][:, ic]
    return BlockInv(lo, hi, ic, ainv, w)


def block_update(h: np.ndarray, inv: BlockInv) -> None:
    """One application of eq. IBMI with I = [lo, hi), in place on H.

    With T = H[I^c, I^c] (the current approximation of the inverse Schur
    complement, taken from the most recent iterate):
      H[I, I^c] = -A_I^{-1} A_{I,I^c} T
      H[I^c, I] = (H[I, I^c])^T
      H[I, I]   = A_I^{-1} + A_I^{-1} A_{I,I^c} T A_{I^c,I} A_I^{-1}
      H[I^c, I^c] = T (unchanged).
    """
    I = np.arange(inv.lo, inv.hi)
    ic = inv.ic
    T = h[np.ix_(ic, ic)]
    X = -(inv.w @ T)
    S = inv.ainv - X @ inv.w.T
    h[np.ix_(I, ic)] = X
    h[np.ix_(ic, I)] = X.T
    h[np.ix_(I, I)] = 0.5 * (S + S.T)


def schur_initial_guess(a: np.ndarray, sets) -> np.ndarray:
    """Initial iterate whose block on the complement of the first set is
    A_{I_1^c}^{-1}, one of the initial guesses of Section 5.6 (Table 6); the
    rest is the identity (only H[I_1^c, I_1^c] is read before it is
    rewritten, Section 2.4)."""
    p = a.shape[0]
    h = np.eye(p)
    ic = complement(p, *sets[0])
    if len(ic):
        h[np.ix_(ic, ic)] = spd_inverse(a[np.ix_(ic, ic)])
    return h


# --------------------------------------------------------------- errors ----

def residual_f(a: np.ndarray, h: np.ndarray) -> float:
    """||I - A H||_F / sqrt(p)."""
    p = a.shape[0]
    R = np.eye(p) - a @ h
    return float(np.sqrt(np.sum(R * R)) / math.sqrt(p))


def paper_error(a: np.ndarray, h: np.ndarray, lo: int, hi: int) -> float:
    """Error estimate of eq. error: the spectral norm of the (1,2) block of
    H A for the set I = [lo, hi), i.e. ||H_I A_{I,I^c} + H_{I,I^c} A_{I^c}||_2."""
    p = a.shape[0]
    ic = complement(p, lo, hi)
    blk = h[lo:hi, lo:hi] @ a[lo:hi][:, ic] + h[lo:hi][:, ic] @ a[np.ix_(ic, ic)]
    return float(np.linalg.norm(blk, 2))


# -------------------------------------------------------- Newton-Schulz ----

def newton_schulz_step(a: np.ndarray, x: np.ndarray):
    """One step of eq. newton, X <- X (2I - A X), written as X + X R with
    R = I - A X; the result is symmetrised.  Returns (X_next, ||R||_F)."""
    p = a.shape[0]
    R = np.eye(p) - a @ x
    xn = x + x @ R
    return 0.5 * (xn + xn.T), float(np.sqrt(np.sum(R * R)))


# ------------------------------------------------------------ Algorithm 1 --

@dataclass
class IbmiResult:
    h: np.ndarray
    status: str                 # "converged" | "not_converged" | "not_spd" | "ns_diverged"
    sweeps: int = 0
    ns_steps: int = 0
    resid_f: float = float("nan")       # last ||I - A H||_F / sqrt(p)
    paper_est: float = float("nan")     # last eq. error estimate (set I_K)
    bad_block: int = -1
    bad_pivot: int = -1
    history: list = field(default_factory=list)


def ibmi(a: np.ndarray, sets, tol: float, max_sweeps: int = 500, h0: np.ndarray | None = None,
         stop_rule: str = "resid_f", check_every: int = 1, ns_theta: float = 0.0,
         ns_max: int = 20) -> IbmiResult:
    """Algorithm 1 with the stopping test of eq. error (or the residual), and
    the optional Newton-Schulz tail of eq. newton.

    h0: initial iterate; only its I_1^c block (the initial approximation of the
    inverse Schur complement) is read.  None means the identity (Section 2.4).
    The stop test runs after every `check_every`-th sweep and after the last
    allowed sweep.  ns_theta > 0 hands over to Newton-Schulz once the unscaled
    ||I - A H||_F <= ns_theta.
    """
    a = np.asarray(a, dtype=np.float64)
    p = a.shape[0]
    h = np.eye(p) if h0 is None else np.array(h0, dtype=np.float64, copy=True)
    invs = []
    for k, (lo, hi) in enumerate(sets):
        try:
            invs.append(block_invariants(a, lo, hi))
        except NotSPD as e:
            return IbmiResult(h, "not_spd", bad_block=k, bad_pivot=lo + e.pivot)
    res = IbmiResult(h, "not_converged")
    lo_K, hi_K = sets[-1]
    r = 0
    while True:
        r += 1
        for inv in invs:
            block_update(h, inv)
        res.sweeps = r
        if r % check_every != 0 and r < max_sweeps:
            continue
        rf = residual_f(a, h)
        res.resid_f = rf
        if stop_rule == "paper":
            res.paper_est = paper_error(a, h, lo_K, hi_K)
            stop_val = res.paper_est
        else:
            stop_val = rf
        res.history.append((r, rf, res.paper_est))
        if not math.isfinite(rf):
            res.status = "nonfinite"
            return res
        if stop_val <= tol:
            res.status = "converged"
            return res
        if ns_theta > 0.0 and rf * math.sqrt(p) <= ns_theta:
            break
        if r >= max_sweeps:
            return res
    # Newton-Schulz tail (eq. newton) on the full iterate.
    prev = res.resid_f
    for s in range(ns_max):
        hn, _ = newton_schulz_step(a, h)
        rf = residual_f(a, hn)
        res.ns_steps = s + 1
        res.history.append(("ns", s + 1, rf))
        if not (rf <= prev):
            res.status = "ns_diverged"
            res.h = h
            return res
        h = hn
        res.h = h
        res.resid_f = prev = rf
        if rf <= tol:
            res.status = "converged"
            return res
    res.status = "not_converged"
    return res


# ---------------------------------------------- partial (block-diagonal) ----

@dataclass
class BlockDiagResult:
    d1: np.ndarray              # H[I_1, I_1]
    d2: np.ndarray              # H[I_2, I_2]
    status: str                 # "converged" | "not_converged" | "nonfinite"
    sweeps: int = 0
    resid_rows: float = float("nan")   # ||(H A - I)[I_2, :]||_F / sqrt(p), last evaluated


def ibmi_block_diagonal(a: np.ndarray, sets, tol: float, max_sweeps: int = 500, t0=None,
                        check_every: int = 1) -> BlockDiagResult:
    """The diagonal blocks of the IBMI iterate alone, for two sets (the partial
    inverse the Discussion of Section 6 proposes).  The step for I_1 reads
    T = H[I_1^c, I_1^c], which lies inside H[I_2, I_2]; the step for I_2 reads
    H[I_2^c, I_2^c], inside H[I_1, I_1] as just rewritten (eq. IBMI), so the
    two blocks evolve on their own.  t0: initial H[I_2, I_2] (only its part on
    I_1^c is read), identity if None.  The stop quantity is the last set's
    rows of the residual, from H[I_2, :] = [X_2 | D_2]; afterwards the overlap
    rows and columns of D_1 take what the last step for I_2 wrote there, as in
    the full iterate."""
    (l1, h1), (l2, h2) = sets
    a = np.asarray(a, dtype=np.float64)
    p = a.shape[0]
    if len(sets) != 2 or l1 != 0 or h2 != p or l2 > h1:
        raise ValueError("two sets covering [0, p)")
    inv1, inv2 = block_invariants(a, l1, h1), block_invariants(a, l2, h2)
    ov = h1 - l2
    d1 = np.eye(h1 - l1)
    d2 = np.eye(h2 - l2) if t0 is None else np.array(t0, dtype=np.float64, copy=True)
    res = BlockDiagResult(d1, d2, "not_converged")
    x2 = None
    r = 0
    while True:
        r += 1
        t1 = d2[ov:, ov:]                        # H[I_1^c, I_1^c]
        x1 = -(inv1.w @ t1)
        s1 = inv1.ainv - x1 @ inv1.w.T
        d1 = 0.5 * (s1 + s1.T)
        t2 = d1[:l2, :l2]                        # H[I_2^c, I_2^c]
        x2 = -(inv2.w @ t2)
        s2 = inv2.ainv - x2 @ inv2.w.T
        d2 = 0.5 * (s2 + s2.T)
        res.sweeps = r
        if r % check_every != 0 and r < max_sweeps:
            continue
        rows = np.hstack([x2, d2])               # H[I_2, :] (columns I_2^c = [0, l2) first)
        R = rows @ a - np.eye(p)[l2:h2]
        res.resid_rows = float(np.sqrt(np.sum(R * R)) / math.sqrt(p))
        if not math.isfinite(res.resid_rows):
            res.status = "nonfinite"
            break
        if res.resid_rows <= tol:
            res.status = "converged"
            break
        if r >= max_sweeps:
            break
    d1 = d1.copy()
    d1[l2:h1, :l2] = x2[:ov]
    d1[:l2, l2:h1] = x2[:ov].T
    d1[l2:h1, l2:h1] = d2[:ov, :ov]
    res.d1, res.d2 = d1, d2
    return res


# ---------------------------------------------------------- flop counts ----

def plan_flops(p: int, sets) -> float:
    """Algorithmic flops of the per-set invariants: Cholesky + inverse
    (m^3/3 + 2 m^3 as counted in Section 4) and A_I^{-1} A_{I,I^c} (2 m^2 n)."""
    f = 0.0
    for lo, hi in sets:
        m = hi - lo
        n = p - m
        f += m ** 3 / 3.0 + 2.0 * m ** 3 + 2.0 * m * m * n
    return f


def sweep_flops(p: int, sets) -> float:
    """Algorithmic flops of one sweep: per set, W T (2 m n^2) and X W^T (2 m^2 n)."""
    f = 0.0
    for lo, hi in sets:
        m = hi - lo
        n = p - m
        f += 2.0 * m * n * n + 2.0 * m * m * n
    return f
