"""Batched inversion and the continuous-batching server vs the FP64 oracle.

The batched entry runs matrices of order <= 2048 as device groups in
lockstep by default (device_batch = 1); the single-matrix pipeline serves the
rest, the fallbacks and every matrix with device_batch = 0.

Matrices whose condition number puts the FP64 floor of ||I - A H||_F/sqrt(p)
(about eps_64 * kappa) above the 1e-10 tolerance cannot reach it in any FP64
arithmetic -- the oracle's Newton-Schulz tail stalls there too.  For those the
check is that the GPU reaches the oracle's own final residual within 5x.
"""
import threading
import time

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


@pytest.fixture(scope="module")
def batch():
    mats = wl.c4_batch(n=16, seed=40, p_max=512)
    mats += [wl.matern32(wl.uniform_points(np.random.default_rng(s), p, 2), 0.1, 1.0, 1e-2)
             for s, p in [(1, 100), (2, 250), (3, 333)]]          # orders off the 64-grid
    refs = []
    for A in mats:
        p = A.shape[0]
        K = 2 if p <= 256 else 3
        h = max(4, round(0.1 * (p // K)))
        refs.append(O.ibmi(A, O.partition(p, K, h), tol=1e-10, max_sweeps=300, ns_theta=0.5))
    return mats, refs


def _run_batched(ibmi, mats, **opts):
    As = [torch.from_numpy(A).cuda() for A in mats]
    Hs = [torch.empty_like(a) for a in As]
    s, res = ibmi.ibmi_invert_batched(As, Hs, **opts)
    torch.cuda.synchronize()
    return s, res, [h.cpu().numpy() for h in Hs]


def _check(A, H, res, ref):
    rf = O.residual_f(A, H)
    if res["status"] == 0:
        # the reported residual is that of the returned H, within 1% of tol
        # (the truncation a correction of the last exact residual is allowed)
        # and the FP64 rounding of the oracle's own product
        assert res["resid_f"] == pytest.approx(rf, rel=1e-2, abs=1e-12), (A.shape, rf, res)
    if ref.status == "converged":
        assert rf <= 1e-10, (A.shape, rf, res)
        inv = np.linalg.inv(A)
        assert np.abs(H - inv).max() <= 1e-6 * np.abs(inv).max()
    else:
        assert rf <= max(1e-10, 5 * ref.resid_f), (A.shape, rf, ref.resid_f, res)
    assert np.array_equal(H, H.T)


def test_batched_mixed_vs_oracle(ibmi, batch):
    mats, refs = batch
    s, res, Hs = _run_batched(ibmi, mats, workers=8)
    for A, H, r, ref in zip(mats, Hs, res, refs):
        _check(A, H, r, ref)
        if ref.status == "converged":
            assert r["status"] == ibmi.IBMI_OK


def test_batched_alone_equals_in_mix(ibmi, batch):
    """Each result is the same whether the matrix runs alone or among others."""
    mats, _ = batch
    _, _, H8 = _run_batched(ibmi, mats, workers=8)
    for i in (0, 5, 17):
        _, _, H1 = _run_batched(ibmi, [mats[i]], workers=1)
        assert np.array_equal(H1[0], H8[i])


def test_batched_graphs_equal_direct_launches(ibmi, batch):
    """Replayed CUDA graphs give the bits the direct launches give, on the
    first call (capture) and on a repeated call (replay of pooled plans)."""
    mats, _ = batch
    sub = [mats[i] for i in (0, 3, 9, 16, 18)]
    _, r0, H0 = _run_batched(ibmi, sub, workers=2, autotune=0, graphs=0)
    for _ in range(2):
        _, r1, H1 = _run_batched(ibmi, sub, workers=2, autotune=0, graphs=1)
        for a, b, x, y in zip(H0, H1, r0, r1):
            assert np.array_equal(a, b)
            assert x["sweeps"] == y["sweeps"] and x["ns_steps"] == y["ns_steps"]
    ibmi.ibmi_batch_release()
    _, _, H2 = _run_batched(ibmi, sub, workers=2, autotune=0, graphs=1)
    for a, b in zip(H0, H2):
        assert np.array_equal(a, b)


def test_batched_fp64(ibmi, batch):
    mats, refs = batch
    sel = [i for i, r in enumerate(refs) if r.status == "converged"][:4]
    s, res, Hs = _run_batched(ibmi, [mats[i] for i in sel], workers=4, precision=ibmi.IBMI_FP64, autotune=0)
    for i, H, r in zip(sel, Hs, res):
        assert r["status"] == ibmi.IBMI_OK
        assert O.residual_f(mats[i], H) <= 1e-10


def test_batched_empty_and_invalid(ibmi):
    s, res = ibmi.ibmi_invert_batched([], [])
    assert s == ibmi.IBMI_OK and res == []


def test_serve_results_alone_and_in_mix(ibmi, batch):
    mats, refs = batch
    srv = ibmi.Server(8 << 30, workers=6)
    rid = srv.submit(mats[3])
    while True:
        st, H_alone, r = srv.poll(rid, mats[3].shape[0])
        if st != ibmi.IBMI_NOT_READY:
            break
        time.sleep(0.002)
    ids = [(i, srv.submit(A)) for i, A in enumerate(mats)]
    out = {}
    t_end = time.time() + 120
    while len(out) < len(ids) and time.time() < t_end:
        for i, rid in ids:
            if i in out:
                continue
            st, H, r = srv.poll(rid, mats[i].shape[0])
            if st != ibmi.IBMI_NOT_READY:
                out[i] = (st, H, r)
        time.sleep(0.002)
    stats = srv.stats()
    srv.close()
    assert len(out) == len(ids)
    assert np.array_equal(out[3][1], H_alone)
    for i, (st, H, r) in out.items():
        _check(mats[i], H, r, refs[i])
    assert stats["completed"] == len(ids) + 1 and stats["p99_s"] >= stats["p50_s"] > 0


def test_serve_admission_respects_budget(ibmi, batch):
    mats, _ = batch
    p = 512
    per_req = 16 * (p * p + p * p)              # bytes charged per request of order 512
    budget = int(per_req * 2.5 / 0.25)          # a quarter of it admits two requests
    srv = ibmi.Server(budget, workers=8)
    big = [A for A in mats if A.shape[0] == p][:1] * 8
    if not big:
        pytest.skip("no p = 512 matrix in the batch")
    ids = [srv.submit(A) for A in big]
    peak = 0
    done = set()
    t_end = time.time() + 120
    while len(done) < len(ids) and time.time() < t_end:
        peak = max(peak, srv.stats()["bytes_in_use"])
        for rid in ids:
            if rid not in done and srv.poll(rid, p)[0] != ibmi.IBMI_NOT_READY:
                done.add(rid)
        time.sleep(0.0005)
    srv.close()
    assert len(done) == len(ids)
    assert peak <= 2 * per_req


def test_serve_cancel_and_budget_reject(ibmi, batch):
    mats, _ = batch
    srv = ibmi.Server(64 << 20, workers=1)    # 64 MB, 16 MB of it for requests
    with pytest.raises(ibmi.IbmiError) as e:
        srv.submit(np.eye(2048))                # 2048^2 * 32 bytes > budget
    assert e.value.status == ibmi.IBMI_ERR_BUDGET
    small = [A for A in mats if A.shape[0] <= 256][:4]
    ids = [srv.submit(A) for A in small]
    assert srv.cancel(ids[-1]) in (ibmi.IBMI_OK, ibmi.IBMI_NOT_READY)
    t_end = time.time() + 60
    pending = set(ids)
    while pending and time.time() < t_end:
        for rid, A in zip(ids, small):
            if rid in pending:
                st, H, r = srv.poll(rid, A.shape[0])
                if st != ibmi.IBMI_NOT_READY:
                    pending.discard(rid)
        time.sleep(0.002)
    srv.close()
    assert not pending


def test_device_groups_match_the_single_matrix_pipeline(ibmi, batch):
    """The lockstep device groups (default) and the per-matrix pipeline
    (device_batch=0) both converge on every matrix, to the same inverse."""
    mats, refs = batch
    _, r1, H1 = _run_batched(ibmi, mats, workers=8)
    _, r0, H0 = _run_batched(ibmi, mats, workers=8, device_batch=0)
    for A, a, b, x, y, ref in zip(mats, H1, H0, r1, r0, refs):
        if ref.status != "converged":
            continue
        assert x["status"] == ibmi.IBMI_OK and y["status"] == ibmi.IBMI_OK, (A.shape, x, y)
        sc = np.abs(b).max()
        assert np.abs(a - b).max() <= 1e-8 * sc, A.shape


@pytest.fixture(scope="module")
def large_batch():
    """The upper buckets of the 512-matrix workload (orders 576..1024)."""
    rng = np.random.default_rng(41)
    mats = []
    for p in (576, 640, 768, 896, 960, 1024, 1024, 768):
        ell = float(np.exp(rng.uniform(np.log(0.05), np.log(0.5))))
        mats.append(wl.squared_exp(wl.uniform_points(rng, p, 3), ell, 1.0, 1e-3))
    refs = []
    for A in mats:
        p = A.shape[0]
        refs.append(O.ibmi(A, O.partition(p, 4, max(4, round(0.1 * (p // 4)))), tol=1e-10, max_sweeps=300,
                           ns_theta=0.5))
    return mats, refs


def test_batched_upper_buckets_vs_oracle(ibmi, large_batch):
    mats, refs = large_batch
    s, res, Hs = _run_batched(ibmi, mats, workers=4)
    for A, H, r, ref in zip(mats, Hs, res, refs):
        _check(A, H, r, ref)
        print(A.shape[0], r["sweeps"], r["ns_steps"], f"{r['resid_f']:.2e}", "oracle", ref.sweeps, ref.ns_steps)


def test_unfinished_matrices_fall_back_and_rerun(ibmi, batch):
    """Without Newton-Schulz steps the sweeps' accuracy floor keeps rho_F
    above 1e-10: every path gives up (the device group, the tuned
    single-matrix run, and the robust rerun where its partition differs) and
    the result is NOT_CONVERGED with the sweeps of all attempts."""
    mats, _ = batch
    sub = [mats[i] for i in (1, 4)]
    s, res, Hs = _run_batched(ibmi, sub, workers=2, ns_max=0, max_sweeps=12)
    assert s == ibmi.IBMI_NOT_CONVERGED
    st = ibmi.ibmi_batch_last_stats()
    assert st["device_matrices"] == 2 and st["fallbacks"] == 2, st
    for r, A, H in zip(res, sub, Hs):
        assert r["status"] == ibmi.IBMI_NOT_CONVERGED and r["sweeps"] >= 2 * 12, r
        assert np.all(np.isfinite(H)) and O.residual_f(A, H) < 1.0


def _kms_inverse(p, rho):
    inv = np.zeros((p, p))
    c = 1.0 / (1.0 - rho * rho)
    i = np.arange(p)
    inv[i, i] = c * (1.0 + rho * rho)
    inv[0, 0] = inv[p - 1, p - 1] = c
    inv[i[:-1], i[:-1] + 1] = inv[i[:-1] + 1, i[:-1]] = -rho * c
    return inv


@pytest.mark.parametrize("family,p", [("kms", 2048), ("matern", 3000), ("cs", 4096)])
def test_serve_families_of_the_trace_at_large_orders(ibmi, family, p):
    """One request of each family of the served trace at orders 2048-4096,
    through the server, against the closed forms (KMS tridiagonal inverse,
    Sherman-Morrison for compound symmetry) or LAPACK (Matern), and the
    oracle's residual."""
    if family == "kms":
        A, inv = wl.kms(p, 0.95), _kms_inverse(p, 0.95)
    elif family == "cs":
        a, b = 0.5, 1.0
        A = wl.compound_symmetry(p, a, b)
        inv = (np.eye(p) - b / (a + p * b) * np.ones((p, p))) / a
    else:
        A = wl.matern32(wl.uniform_points(np.random.default_rng(9), p, 2), 0.1, 1.0, 1e-2)
        inv = np.linalg.inv(A)
    srv = ibmi.Server(64 << 30, workers=4)
    rid = srv.submit(A)
    t_end = time.time() + 300
    while time.time() < t_end:
        st, H, r = srv.poll(rid, p)
        if st != ibmi.IBMI_NOT_READY:
            break
        time.sleep(0.005)
    srv.close()
    assert st == ibmi.IBMI_OK, (family, r)
    rf = O.residual_f(A, H)
    print(f"{family} p={p}: {r['sweeps']} sweeps + {r['ns_steps']} NS, rho_F {rf:.2e}")
    assert rf <= 1e-10
    assert np.abs(H - inv).max() <= 1e-8 * np.abs(inv).max()
