"""The seeded synthetic inputs follow the recipes stated for the benchmark
configurations (shapes, value ranges, distributions), and the same seed gives
the same input on every machine."""
import math

import numpy as np
import pytest

import workloads as wl


def _spd(a):
    np.linalg.cholesky(a)   # raises if not positive definite
    return True


def test_kms_and_compound_symmetry_definitions():
    p, rho = 9, 0.7
    a = wl.kms(p, rho)
    i, j = np.indices((p, p))
    np.testing.assert_array_equal(a, rho ** np.abs(i - j))
    c = wl.compound_symmetry(p, 0.5, 0.25)
    np.testing.assert_array_equal(c, 0.5 * np.eye(p) + 0.25 * np.ones((p, p)))


def test_c2_matern_recipe_and_determinism():
    a = wl.c2_matern(p=256, seed=2)
    assert a.shape == (256, 256) and np.array_equal(a, a.T)
    np.testing.assert_allclose(np.diag(a), 1.0 + 1e-2, rtol=0, atol=1e-15)   # unit variance + nugget
    off = a[~np.eye(256, dtype=bool)]
    assert off.min() > 0.0 and off.max() < 1.0
    assert _spd(a)
    assert np.array_equal(a, wl.c2_matern(p=256, seed=2))
    assert not np.array_equal(a, wl.c2_matern(p=256, seed=3))


def test_c3_random_spd_spectrum():
    a = wl.c3_random_spd(p=256, seed=3)
    assert np.array_equal(a, a.T)
    lam = np.linalg.eigvalsh(a)
    assert lam.min() >= 1.0 - 1e-9 and lam.max() <= 1e4 * (1 + 1e-9)
    # log-uniform: about half of the eigenvalues below 100
    assert 0.35 < np.mean(lam < 100.0) < 0.65


def test_c4_batch_sizes_and_matrices():
    mats = wl.c4_batch(n=24, seed=4)
    sizes = [m.shape[0] for m in mats]
    assert all(s % 64 == 0 and 64 <= s <= 1024 for s in sizes)
    assert len(set(sizes)) > 5
    for m in mats[:6]:
        assert np.array_equal(m, m.T)
        np.testing.assert_allclose(np.diag(m), 1.0 + 1e-3, rtol=0, atol=1e-15)
        assert _spd(m)
    again = wl.c4_batch(n=24, seed=4)
    assert all(np.array_equal(x, y) for x, y in zip(mats, again))


def test_c5_trace_rate_sizes_and_families():
    tr = wl.c5_trace(2.0, rate=2000.0, seed=5)
    assert 0.9 * 4000 < len(tr) < 1.1 * 4000
    ts = [r.t_arrival for r in tr]
    assert ts == sorted(ts) and ts[-1] < 2.0
    ps = np.array([r.p for r in tr])
    assert ps.min() >= 128 and ps.max() <= 4096
    # log-uniform: the median order near sqrt(128 * 4096) = 724
    assert 600 < np.median(ps) < 870
    fams = [r.family for r in tr]
    for f in ("kms", "matern", "cs"):
        assert abs(fams.count(f) / len(fams) - 1 / 3) < 0.05
    for r in tr:
        if r.family == "kms":
            assert 0.1 <= r.params[0] <= 0.95
        elif r.family == "cs":
            assert 0.5 <= r.params[0] <= 2.0 and 0.0 <= r.params[1] <= 1.0
    small = [r for r in tr if r.p <= 200][:3]
    for r in small:
        m = r.matrix(seed=11)
        assert m.shape == (r.p, r.p) and _spd(m)
