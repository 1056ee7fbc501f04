"""The allocation-free residual entry point, through the C ABI.

ibmi_residual_noalloc serves callers that cannot call cudaMalloc (code under
an external device-memory manager, latency-critical loops where an allocation
may synchronise the device); it keeps its scratch in a fixed array inside the
library.  Two calls in a row, with different orders, must both agree with the
allocating ibmi_residual to FP64 rounding (the same kernels run on the same
data; only where the partial sums live differs), which also shows that the
second call is not affected by what the first left in the shared scratch.
This file is collected last so that a failure here never hides another test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2502_06377_gb300 import _lib
    return _lib.load()


def _resid(lib, fn, A, H):
    out = C.c_double()
    s = getattr(lib, fn)(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(H.data_ptr()), H.stride(0),
                         A.shape[0], None, C.byref(out))
    assert s == 0, (fn, s, lib.ibmi_last_error())
    return out.value


def test_noalloc_residual_matches_allocating_entry(lib):
    results = []
    for p, seed in ((700, 1), (4096, 2)):          # two calls in a row, different orders
        rng = np.random.default_rng(seed)
        A = wl.matern32(wl.uniform_points(rng, p, 2), 0.1, 1.0, 1e-2)
        H = np.linalg.inv(A) + 1e-7 * rng.standard_normal((p, p))
        dA, dH = torch.from_numpy(A).cuda(), torch.from_numpy(H).cuda()
        got = _resid(lib, "ibmi_residual_noalloc", dA, dH)
        ref = _resid(lib, "ibmi_residual", dA, dH)
        assert got == pytest.approx(ref, rel=1e-12, abs=1e-15)
        results.append(got)
    assert results[0] != results[1]


def test_noalloc_residual_matches_the_oracle_and_reads_the_lower_triangle(lib):
    """Against the FP64 oracle's ||I - A H||_F / sqrt(p), with NaN in the
    strict upper triangle of A (only the lower triangle may be read), two
    calls in a row."""
    from oracle import ibmi_oracle as O
    for p, seed in ((333, 3), (1000, 4)):
        rng = np.random.default_rng(seed)
        A = wl.matern32(wl.uniform_points(rng, p, 2), 0.1, 1.0, 1e-2)
        H = np.linalg.inv(A) + 1e-8 * rng.standard_normal((p, p))
        want = O.residual_f(A, H)
        An = A.copy()
        An[np.triu_indices(p, 1)] = np.nan
        dA, dH = torch.from_numpy(An).cuda(), torch.from_numpy(H).cuda()
        got = _resid(lib, "ibmi_residual_noalloc", dA, dH)
        assert got == pytest.approx(want, rel=1e-9)


def test_noalloc_rejects_orders_beyond_its_scratch(lib):
    A = torch.empty((1, 1), dtype=torch.float64, device="cuda")
    out = C.c_double()
    s = lib.ibmi_residual_noalloc(C.c_void_p(A.data_ptr()), 8193, C.c_void_p(A.data_ptr()), 8193, 8193, None,
                                  C.byref(out))
    assert s == 1 and b"8192" in lib.ibmi_last_error()
