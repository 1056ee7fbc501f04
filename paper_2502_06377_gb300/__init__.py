"""GB300-native IBMI (Iterative Block Matrix Inversion) block-sweep inverter.

The compute path is the CUDA library libibmi.so behind the C ABI declared in
include/ibmi.h; this package is its thin Python binding.  Functions keep the
C names and take torch CUDA tensors (or numpy arrays for the *_host variants)
in place of raw pointers.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (IBMI_FP64, IBMI_MIXED, IBMI_INIT_IDENTITY, IBMI_INIT_USER, IBMI_INIT_SCHUR,  # noqa: F401
                   IBMI_STOP_RESID_F, IBMI_STOP_PAPER_EST, IBMI_OK, IBMI_NOT_CONVERGED,
                   IBMI_ERR_NOT_SPD, IBMI_ERR_INVALID_ARG, IBMI_ERR_NONFINITE, IBMI_ERR_OOM,
                   IBMI_ERR_TIMEOUT, IBMI_ERR_CUDA, ibmi_plan_desc, ibmi_result)


class IbmiError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        lib = _lib.load()
        msg = lib.ibmi_status_string(status).decode()
        err = lib.ibmi_last_error().decode()
        super().__init__(f"{what}: {msg}" + (f" ({err})" if err else ""))
        self.status = status


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def ibmi_plan_desc_init(**kw) -> ibmi_plan_desc:
    d = ibmi_plan_desc()
    _lib.load().ibmi_plan_desc_init(C.byref(d))
    for k, v in kw.items():
        if k in ("lo", "hi"):
            continue
        setattr(d, k, v)
    return d


class Plan:
    """Owns an ibmi_plan_t; the explicit set arrays are kept alive here."""

    def __init__(self, desc: ibmi_plan_desc, lo=None, hi=None):
        self._lib = _lib.load()
        self._keep = []
        if lo is not None:
            lo_a = (C.c_int64 * len(lo))(*[int(v) for v in lo])
            hi_a = (C.c_int64 * len(hi))(*[int(v) for v in hi])
            self._keep += [lo_a, hi_a]
            desc.lo = C.cast(lo_a, C.POINTER(C.c_int64))
            desc.hi = C.cast(hi_a, C.POINTER(C.c_int64))
            desc.K = len(lo)
        self.desc = desc
        h = C.c_void_p()
        s = self._lib.ibmi_plan(C.byref(desc), C.byref(h))
        if s != IBMI_OK:
            raise IbmiError(s, "ibmi_plan")
        self.handle = h

    def sets(self):
        K = C.c_int32()
        self._lib.ibmi_plan_sets(self.handle, C.byref(K), None, None)
        lo = (C.c_int64 * K.value)()
        hi = (C.c_int64 * K.value)()
        self._lib.ibmi_plan_sets(self.handle, None, lo, hi)
        return list(zip(list(lo), list(hi)))

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ibmi_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ibmi_plan(p: int, K: int = 2, h: int = 0, lo=None, hi=None, **kw) -> Plan:
    return Plan(ibmi_plan_desc_init(p=p, K=K, h=h, **kw), lo, hi)


def ibmi_invert(plan: Plan, A, H, stream=None):
    """A, H: torch float64 CUDA tensors (p x p, row stride >= p).  Returns
    (status, result dict)."""
    assert A.dtype == H.dtype and str(A.dtype) == "torch.float64" and A.is_cuda and H.is_cuda
    assert A.stride(1) == 1 and H.stride(1) == 1
    res = ibmi_result()
    s = _lib.load().ibmi_invert(plan.handle, C.c_void_p(A.data_ptr()), A.stride(0),
                                C.c_void_p(H.data_ptr()), H.stride(0), _stream_ptr(stream), C.byref(res))
    return s, res.as_dict()


def ibmi_invert_block_diag(plan: Plan, A, D, stream=None):
    """Diagonal blocks of the iterate for a two-set plan: D is a float64 CUDA
    tensor of m_1^2 + m_2^2 elements (H[I_1, I_1] then H[I_2, I_2], row-major).
    Returns (status, result dict)."""
    assert str(A.dtype) == "torch.float64" and A.is_cuda and A.stride(1) == 1
    assert str(D.dtype) == "torch.float64" and D.is_cuda and D.is_contiguous()
    res = ibmi_result()
    s = _lib.load().ibmi_invert_block_diag(plan.handle, C.c_void_p(A.data_ptr()), A.stride(0),
                                           C.c_void_p(D.data_ptr()), _stream_ptr(stream), C.byref(res))
    return s, res.as_dict()


def ibmi_invert_host(plan: Plan, A: np.ndarray, H: np.ndarray, stream=None):
    """A, H: C-contiguous float64 numpy arrays (ideally pinned)."""
    assert A.dtype == np.float64 and H.dtype == np.float64
    assert A.flags.c_contiguous and H.flags.c_contiguous
    res = ibmi_result()
    s = _lib.load().ibmi_invert_host(plan.handle, C.c_void_p(A.ctypes.data), A.shape[1],
                                     C.c_void_p(H.ctypes.data), H.shape[1], _stream_ptr(stream),
                                     C.byref(res))
    return s, res.as_dict()


def ibmi_residual(A, H, stream=None) -> float:
    out = C.c_double()
    s = _lib.load().ibmi_residual(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(H.data_ptr()),
                                  H.stride(0), A.shape[0], _stream_ptr(stream), C.byref(out))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_residual")
    return out.value


def ibmi_status_string(s: int) -> str:
    return _lib.load().ibmi_status_string(s).decode()


def ibmi_residual_noalloc(A, H, stream=None) -> float:
    """ibmi_residual without device allocation (fixed library scratch, p <= 8192)."""
    out = C.c_double()
    s = _lib.load().ibmi_residual_noalloc(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(H.data_ptr()),
                                          H.stride(0), A.shape[0], _stream_ptr(stream), C.byref(out))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_residual_noalloc")
    return out.value


def ibmi_selftest_wait_timeout(stream=None) -> int:
    """Runs the bounded-wait self-test launch; returns its status
    (IBMI_ERR_TIMEOUT is the intended outcome)."""
    return _lib.load().ibmi_selftest_wait_timeout(_stream_ptr(stream))


def ibmi_residual_tc(A, H, stream=None) -> float:
    """FP64-accurate ||I - A H||_F / sqrt(p) on tensor cores (sliced error-free products)."""
    out = C.c_double()
    s = _lib.load().ibmi_residual_tc(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(H.data_ptr()),
                                     H.stride(0), A.shape[0], _stream_ptr(stream), C.byref(out))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_residual_tc")
    return out.value


def ibmi_refine(A, X, precision=IBMI_MIXED, tol=1e-10, ns_max=8, stream=None):
    """Newton-Schulz refinement of the symmetric approximate inverse X (in place)."""
    res = ibmi_result()
    s = _lib.load().ibmi_refine(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(X.data_ptr()), X.stride(0),
                                A.shape[0], precision, tol, ns_max, _stream_ptr(stream), C.byref(res))
    return s, res.as_dict()


# ------------------------------------------------- orderings and tuning --

from ._lib import (IBMI_ORDER_IDENTITY, IBMI_ORDER_XSORT, IBMI_ORDER_HILBERT, IBMI_ORDER_KD,  # noqa: E402,F401
                   IBMI_ORDER_REDBLACK, ibmi_tune_candidate)


def ibmi_order_points(points: np.ndarray, order: int) -> np.ndarray:
    """Permutation (int64, n) placing the points (n x dim) in the given order."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    if pts.ndim == 1:
        pts = pts[:, None]
    perm = np.empty(pts.shape[0], dtype=np.int64)
    s = _lib.load().ibmi_order_points(pts.ctypes.data_as(C.POINTER(C.c_double)), pts.shape[0], pts.shape[1],
                                      order, perm.ctypes.data_as(C.POINTER(C.c_int64)))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_order_points")
    return perm


def ibmi_permute(A, perm, B, inverse: bool = False, stream=None) -> None:
    """B = A[perm][:, perm] (or its inverse) on the device."""
    q = np.ascontiguousarray(perm, dtype=np.int64)
    s = _lib.load().ibmi_permute(C.c_void_p(A.data_ptr()), A.stride(0), A.shape[0],
                                 q.ctypes.data_as(C.POINTER(C.c_int64)), 1 if inverse else 0,
                                 C.c_void_p(B.data_ptr()), B.stride(0), _stream_ptr(stream))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_permute")


def ibmi_tune(A, perms=(), stream=None, **base):
    """Measured search over orderings (the given one and `perms`) and
    partitions; `base` sets the plan options (precision, tol, ...).  Returns
    (status, best candidate dict, list of all candidate dicts)."""
    p = A.shape[0]
    qs = [np.ascontiguousarray(q, dtype=np.int64) for q in perms]
    arr = (C.POINTER(C.c_int64) * max(1, len(qs)))(*[q.ctypes.data_as(C.POINTER(C.c_int64)) for q in qs])
    d = ibmi_plan_desc_init(p=p, **base)
    best = ibmi_tune_candidate()
    cap = 256
    allc = (ibmi_tune_candidate * cap)()
    n = C.c_int32()
    s = _lib.load().ibmi_tune(C.c_void_p(A.data_ptr()), A.stride(0), p, arr, len(qs), C.byref(d),
                              _stream_ptr(stream), C.byref(best), allc, cap, C.byref(n))
    return s, best.as_dict(), [allc[i].as_dict() for i in range(min(n.value, cap))]


# ----------------------------------------------------------------- batches --

from ._lib import ibmi_batch_opts  # noqa: E402

IBMI_NOT_READY = _lib.IBMI_NOT_READY
IBMI_ERR_CANCELLED = _lib.IBMI_ERR_CANCELLED
IBMI_ERR_BUDGET = _lib.IBMI_ERR_BUDGET


def ibmi_batch_opts_init(**kw) -> ibmi_batch_opts:
    o = ibmi_batch_opts()
    _lib.load().ibmi_batch_opts_init(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def ibmi_plan_bytes(p: int, K: int = 2, h: int = 0, **kw) -> int:
    return _lib.load().ibmi_plan_bytes(C.byref(ibmi_plan_desc_init(p=p, K=K, h=h, **kw)))


def ibmi_invert_batched(As, Hs, **opts):
    """As, Hs: lists of torch float64 CUDA tensors (square, row stride >= p).
    Returns (status, [result dict per matrix])."""
    n = len(As)
    P = (C.c_int64 * n)(*[a.shape[0] for a in As])
    LA = (C.c_int64 * n)(*[a.stride(0) for a in As])
    LH = (C.c_int64 * n)(*[h.stride(0) for h in Hs])
    PA = (C.c_void_p * n)(*[a.data_ptr() for a in As])
    PH = (C.c_void_p * n)(*[h.data_ptr() for h in Hs])
    out = (ibmi_result * n)()
    o = ibmi_batch_opts_init(**opts)
    s = _lib.load().ibmi_invert_batched(n, P, PA, LA, PH, LH, C.byref(o), out)
    return s, [out[i].as_dict() for i in range(n)]


def ibmi_batch_last_stats() -> dict:
    """Counters of the last batched call (device groups, rounds, fallbacks, phase seconds)."""
    st = _lib.ibmi_batch_stats()
    s = _lib.load().ibmi_batch_last_stats(C.byref(st))
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_batch_last_stats")
    return st.as_dict()


def ibmi_batch_release() -> None:
    """Frees the pooled batch workers (streams, plans, captured graphs)."""
    s = _lib.load().ibmi_batch_release()
    if s != IBMI_OK:
        raise IbmiError(s, "ibmi_batch_release")


class Server:
    """Continuous-batching inversion server (ibmi_serve_*)."""

    def __init__(self, hbm_budget_bytes: int, **opts):
        self._lib = _lib.load()
        self._opts = ibmi_batch_opts_init(**opts)
        h = C.c_void_p()
        s = self._lib.ibmi_serve_create(int(hbm_budget_bytes), C.byref(self._opts), C.byref(h))
        if s != IBMI_OK:
            raise IbmiError(s, "ibmi_serve_create")
        self.handle = h

    def submit(self, A: np.ndarray, tol: float = 1e-10) -> int:
        A = np.ascontiguousarray(A, dtype=np.float64)
        rid = C.c_uint64()
        s = self._lib.ibmi_serve_submit(self.handle, C.c_void_p(A.ctypes.data), A.shape[0], A.shape[1], tol,
                                        C.byref(rid))
        if s != IBMI_OK:
            raise IbmiError(s, "ibmi_serve_submit")
        return rid.value

    def poll(self, rid: int, p: int):
        """Returns (status, H or None, result dict)."""
        H = np.empty((p, p), dtype=np.float64)
        res = ibmi_result()
        s = self._lib.ibmi_serve_poll(self.handle, rid, C.c_void_p(H.ctypes.data), p, C.byref(res))
        if s == IBMI_NOT_READY or s == IBMI_ERR_CANCELLED:
            return s, None, None
        return s, H, res.as_dict()

    def cancel(self, rid: int) -> int:
        return self._lib.ibmi_serve_cancel(self.handle, rid)

    def stats(self):
        p50, p99, ips = C.c_double(), C.c_double(), C.c_double()
        n, used = C.c_int64(), C.c_uint64()
        self._lib.ibmi_serve_stats(self.handle, C.byref(p50), C.byref(p99), C.byref(ips), C.byref(n),
                                   C.byref(used))
        return {"p50_s": p50.value, "p99_s": p99.value, "inverses_per_s": ips.value, "completed": n.value,
                "bytes_in_use": used.value}

    def reset_stats(self):
        """Forget the latencies and counts so far (e.g. after a warm-up)."""
        self._lib.ibmi_serve_stats_reset(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self._lib.ibmi_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
