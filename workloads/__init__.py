"""Seeded synthetic SPD inputs for the IBMI block-sweep inverter.

This module only draws random numbers and evaluates covariance kernels; it
holds none of the inversion arithmetic.  Both the GPU path and the FP64 oracle
read their inputs from here, so the two always see identical matrices.

Families (covariance kernels of Table 1 and the textbook families used as
closed-form checks):

* ``kms``            -- A_ij = rho^|i-j| (AR(1) / Kac-Murdock-Szego).
* ``compound_symmetry`` -- a I + b 1 1^T.
* ``matern32``       -- Matern 3/2 kernel (Table 1) on seeded points.
* ``squared_exp``    -- RBF / squared-exponential kernel (Table 1).
* ``exp_1d`` / ``iquad_1d`` -- the exponential and inverse-quadratic kernels
  of Table 1 on the 1-D grid of Section 5 (points equally spaced on [0, p^0.9]).
* ``random_spd``     -- Q diag(lambda) Q^T with Q from a QR factorisation.

Random points are sorted by their first coordinate so that the matrix has the
diagonal dominance the partitioned sweep relies on (Section 5, discussion of
the properties that affect convergence).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "kms", "compound_symmetry", "matern32", "squared_exp", "exp_1d", "iquad_1d",
    "random_spd", "uniform_points", "pairwise_dist", "c1_kms", "c2_matern",
    "c3_random_spd", "c4_batch", "c5_trace", "ServeRequest",
]


def kms(p: int, rho: float) -> np.ndarray:
    i = np.arange(p)
    return np.power(float(rho), np.abs(i[:, None] - i[None, :])).astype(np.float64)


def compound_symmetry(p: int, a: float, b: float) -> np.ndarray:
    return a * np.eye(p) + b * np.ones((p, p))


def uniform_points(rng: np.random.Generator, n: int, dim: int, sort: bool = True) -> np.ndarray:
    x = rng.random((n, dim))
    if sort:
        x = x[np.argsort(x[:, 0], kind="stable")]
    return x


def pairwise_dist(x: np.ndarray) -> np.ndarray:
    d2 = ((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    return np.sqrt(np.maximum(d2, 0.0))


def matern32(x: np.ndarray, ell: float, sigma2: float = 1.0, nugget: float = 0.0) -> np.ndarray:
    r = math.sqrt(3.0) * pairwise_dist(x) / ell
    a = sigma2 * (1.0 + r) * np.exp(-r)
    a[np.diag_indices_from(a)] += nugget
    return a


def squared_exp(x: np.ndarray, ell: float, sigma2: float = 1.0, nugget: float = 0.0) -> np.ndarray:
    d = pairwise_dist(x)
    a = sigma2 * np.exp(-(d * d) / (2.0 * ell * ell))
    a[np.diag_indices_from(a)] += nugget
    return a


def _grid_1d(p: int) -> np.ndarray:
    return np.linspace(0.0, float(p) ** 0.9, p)


def exp_1d(p: int) -> np.ndarray:
    x = _grid_1d(p)
    return np.exp(-np.abs(x[:, None] - x[None, :]) / 5.0)


def iquad_1d(p: int) -> np.ndarray:
    x = _grid_1d(p)
    return 1.0 / np.sqrt(1.0 + (x[:, None] - x[None, :]) ** 2)


def random_spd(p: int, seed: int, lam_lo: float = 1.0, lam_hi: float = 1e4) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((p, p))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    lam = np.exp(rng.uniform(math.log(lam_lo), math.log(lam_hi), size=p))
    a = (q * lam[None, :]) @ q.T
    return 0.5 * (a + a.T)


# ---------------------------------------------------------------- workloads --

def c1_kms() -> np.ndarray:
    """p = 256 AR(1) matrix, rho = 0.5 (two-block, non-overlapping case)."""
    return kms(256, 0.5)


def c2_matern(p: int = 4096, seed: int = 2) -> np.ndarray:
    """Matern 3/2 on p seeded points in the unit square, ell = 0.1, unit variance,
    nugget 1e-2, points sorted by x."""
    rng = np.random.default_rng(seed)
    return matern32(uniform_points(rng, p, 2), ell=0.1, sigma2=1.0, nugget=1e-2)


def c3_random_spd(p: int = 8192, seed: int = 3) -> np.ndarray:
    """Q diag(lambda) Q^T, lambda log-uniform in [1, 1e4]."""
    return random_spd(p, seed, 1.0, 1e4)


def c4_batch(n: int = 512, seed: int = 4, p_step: int = 64, p_max: int = 1024):
    """n squared-exponential matrices on seeded 3-D points, p uniform in
    {p_step, 2 p_step, ..., p_max}, length scale log-uniform in [0.05, 0.5],
    nugget 1e-3.  Returns a list of float64 arrays."""
    rng = np.random.default_rng(seed)
    sizes = p_step * rng.integers(1, p_max // p_step + 1, size=n)
    ells = np.exp(rng.uniform(math.log(0.05), math.log(0.5), size=n))
    mats = []
    for p, ell in zip(sizes, ells):
        x = uniform_points(rng, int(p), 3)
        mats.append(squared_exp(x, float(ell), 1.0, 1e-3))
    return mats


@dataclass
class ServeRequest:
    t_arrival: float
    family: str
    p: int
    params: tuple

    def matrix(self, seed: int) -> np.ndarray:
        if self.family == "kms":
            return kms(self.p, self.params[0])
        if self.family == "cs":
            return compound_symmetry(self.p, self.params[0], self.params[1])
        rng = np.random.default_rng(seed)
        return matern32(uniform_points(rng, self.p, 2), ell=0.1, sigma2=1.0, nugget=1e-2)


def c5_trace(duration_s: float, rate: float = 2000.0, seed: int = 5,
             p_lo: int = 128, p_hi: int = 4096) -> list:
    """Poisson arrivals at `rate` per second; p log-uniform in [p_lo, p_hi];
    families KMS (rho ~ U[.1,.95]), Matern 3/2 (as c2_matern), compound symmetry
    (a ~ U[.5,2], b ~ U[0,1]) drawn with equal probability."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        p = int(round(math.exp(rng.uniform(math.log(p_lo), math.log(p_hi)))))
        fam = ("kms", "matern", "cs")[int(rng.integers(0, 3))]
        if fam == "kms":
            params = (float(rng.uniform(0.1, 0.95)),)
        elif fam == "cs":
            params = (float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.0, 1.0)))
        else:
            params = ()
        out.append(ServeRequest(t, fam, p, params))
    return out
