"""Command-line runner for single library calls on cuda:0.

  python -m paper_2502_06377_gb300 invert   --p 4096 --K 8 --h 32 --precision mixed --theta 0.9 --init identity
  python -m paper_2502_06377_gb300 residual --p 4096 --method tc
  python -m paper_2502_06377_gb300 batch    --only-p 1024 --autotune 0 --repeat 2

Inputs are the seeded Matern-3/2 covariance of the benchmark (points in the
unit square sorted by x, length scale 0.1, nugget 1e-2).  `residual` evaluates
||I - A H||_F / sqrt(p) for H = the identity-initialised IBMI result after one
sweep (a realistic iterate).  `batch` inverts the 512 squared-exponential
matrices of the batched workload (seed 4; --only-p keeps the matrices of one
order) with ibmi_invert_batched.  Prints one JSON line.
"""
import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser(prog="python -m paper_2502_06377_gb300")
    ap.add_argument("cmd", choices=["invert", "residual", "batch"])
    ap.add_argument("--p", type=int, default=4096)
    ap.add_argument("--K", type=int, default=8)
    ap.add_argument("--h", type=int, default=32)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--method", choices=["tc", "fp64"], default="tc")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--family", choices=["matern", "random_spd"], default="matern",
                    help="matern: the Matern-3/2 workload; random_spd: Q diag(lambda) Q^T, lambda "
                         "log-uniform in [1, 1e4] (seed 3)")
    ap.add_argument("--max-sweeps", type=int, default=500)
    ap.add_argument("--theta", type=float, default=0.5,
                    help="Newton-Schulz hand-over on ||I - A H||_F (mixed precision)")
    ap.add_argument("--init", choices=["identity", "schur"], default="identity",
                    help="initial iterate: H = I, or T_0 = A_{I_1^c}^{-1} (invert)")
    ap.add_argument("--only-p", type=int, default=0, help="batch: only the matrices of this order")
    ap.add_argument("--autotune", type=int, default=1, help="batch: tune (K, h) per size bucket")
    ap.add_argument("--device-batch", type=int, default=1, help="batch: run device groups")
    a = ap.parse_args()
    if a.cmd == "batch":
        return run_batch(a)

    import numpy as np
    import torch

    from paper_2502_06377_gb300 import build as _b
    _b.build()
    import paper_2502_06377_gb300 as ibmi
    import workloads as wl

    A = wl.c2_matern(a.p, seed=2) if a.family == "matern" else wl.c3_random_spd(a.p, seed=3)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    prec = ibmi.IBMI_MIXED if a.precision == "mixed" else ibmi.IBMI_FP64
    if a.cmd == "invert":
        plan = ibmi.ibmi_plan(a.p, K=a.K, h=a.h, precision=prec, tol=a.tol, max_sweeps=a.max_sweeps,
                              ns_theta=a.theta if prec == ibmi.IBMI_MIXED else 0.0,
                              init=ibmi.IBMI_INIT_SCHUR if a.init == "schur" else ibmi.IBMI_INIT_IDENTITY)
        ibmi._lib.load().ibmi_prof_enable(1)
        out = None
        for _ in range(a.repeat):
            t0 = time.perf_counter()
            s, res = ibmi.ibmi_invert(plan, dA, dH)
            torch.cuda.synchronize()
            out = dict(res, status_name=ibmi.ibmi_status_string(s), wall_s=time.perf_counter() - t0)
        import ctypes as C
        lib = ibmi._lib.load()
        names = ["sweep_x", "sweep_s", "residual", "newton_schulz", "invariants", "other", "invariants_tc"]
        prof, calls = {}, {}
        for k, nm in enumerate(names):
            n, t, f = C.c_int64(), C.c_double(), C.c_double()
            lib.ibmi_prof_get(k, C.byref(n), C.byref(t), C.byref(f))
            prof[nm] = round(t.value / a.repeat, 3)
            calls[nm] = n.value / a.repeat
        out["ms_per_class"] = prof
        out["calls_per_class"] = calls
        print(json.dumps(out))
    else:
        plan = ibmi.ibmi_plan(a.p, K=a.K, h=a.h, precision=ibmi.IBMI_FP64, tol=0.0, max_sweeps=1)
        ibmi.ibmi_invert(plan, dA, dH)
        torch.cuda.synchronize()
        fn = ibmi.ibmi_residual_tc if a.method == "tc" else ibmi.ibmi_residual
        v = None
        for _ in range(a.repeat):
            t0 = time.perf_counter()
            v = fn(dA, dH)
            dt = time.perf_counter() - t0
        print(json.dumps({"resid_f": v, "method": a.method, "p": a.p, "wall_s": dt}))


def run_batch(a):
    import torch

    from paper_2502_06377_gb300 import build as _b
    _b.build()
    import paper_2502_06377_gb300 as ibmi
    import workloads as wl

    mats = [A for A in wl.c4_batch(n=512, seed=4) if not a.only_p or A.shape[0] == a.only_p]
    As = [torch.from_numpy(A).cuda() for A in mats]
    Hs = [torch.empty_like(x) for x in As]
    out = None
    for _ in range(a.repeat):
        t0 = time.perf_counter()
        s, res = ibmi.ibmi_invert_batched(As, Hs, workers=16, autotune=a.autotune, device_batch=a.device_batch,
                                          tol=a.tol)
        torch.cuda.synchronize()
        out = {"status": ibmi.ibmi_status_string(s), "matrices": len(mats), "wall_s": time.perf_counter() - t0,
               "converged": sum(r["status"] == 0 for r in res), "stats": ibmi.ibmi_batch_last_stats()}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
