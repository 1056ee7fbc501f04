#!/usr/bin/env python
"""IBMI inversion benchmark on GB300.

Headline metric: SPD inverses per second at ||I - A H||_F / sqrt(p) <= 1e-10
on the p = 4096 Matern-3/2 workload (4096 seeded points in the unit square
sorted by x, length scale 0.1, unit variance, nugget 1e-2; K = 8 sets of
544/576 rows with 64-row overlap).  One step = one complete inversion through
the C ABI (block invariants, sweeps, stop tests, Newton-Schulz tail), with A
resident in HBM.  A and H are 134 MB each, larger than the 129 MB L2, so no
L2 flush is needed between steps.

The default run (--workload all) also measures, inside the same JSON line
under "configs", the other workloads of the method's scope, each with its
own clock record:
  c3    p = 8192 random SPD (Q diag(lambda) Q^T, lambda log-uniform in
        [1, 1e4]), K = 2, h = 1024, mixed precision from T_0 = A_{I_1^c}^{-1};
        the identity start and one FP64 sweep timed for comparison;
  c4    512 squared-exponential matrices of order 64..1024 through the
        batched entry point, mixed precision, and mixed vs plain FP64 on a
        64-matrix sample of the batch;
  c5    Poisson request traces into the continuous-batching server at three
        offered rates (the 2000 requests/s of the workload and two below
        saturation), p50/p99 latency and drained throughput, and a sample of
        the same requests served in FP64.

--impl reference times the FP64 CPU oracle: each step is one complete
oracle solve of the headline workload (the same partition and hand-over as
the GPU path) on the host cores.

Multi-GPU: every rank inverts its own copy of the headline workload
(independent problems, no collective); value = inverses of all ranks /
max-over-ranks time.  The other configurations run at N = 1 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPD inverses/s @ ||I-AH||_F/sqrt(p)<=1e-10 (p=4096 Matern-3/2, K=8)"
P, K_SETS, H_OV, TOL, THETA = 4096, 8, 32, 1e-10, 0.9
FP64_PEAK_TFLOPS = 1.25   # FP64 (DFMA) peak of GB300, nominal figure for the part
CLASSES = ["sweep_x", "sweep_s", "residual", "newton_schulz", "invariants", "other", "invariants_tc"]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        j = json.load(open(path))
        return {"hbm_gbs": j.get("hbm_gbs"), "bf16": j.get("bf16_tflops"),
                "bf16_sustained": j.get("bf16_tflops_sustained"), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "src": "fallback"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--workload", default="all", choices=["all", "c2", "c3", "batch", "serve"],
                    help="all: the headline line with the other workloads under 'configs'; c2: the "
                         "headline alone; c3 / batch / serve: one of the other workloads alone")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--serve-seconds", type=float, default=0.5)
    ap.add_argument("--serve-rates", default="2000,120,60",
                    help="offered request rates (per second) of the served traces")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [s.strip() for s in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i - 5] for r in self.rows for i in range(5, 9) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ oracle --

def oracle_solve(A, K, h, tol=TOL, theta=THETA):
    """One complete FP64 oracle solve (Algorithm 1 with the Newton-Schulz
    hand-over at ||I - A H||_F <= theta, as the GPU path runs it).  Returns
    (seconds, result)."""
    from oracle import ibmi_oracle as O
    p = A.shape[0]
    t0 = time.perf_counter()
    res = O.ibmi(A, O.partition(p, K, h), tol=tol, max_sweeps=500, ns_theta=theta)
    return time.perf_counter() - t0, res


def vs_oracle(A, H, ref):
    """Error of a GPU result against the oracle's solve of the same input."""
    import numpy as np
    from oracle import ibmi_oracle as O
    d = H - ref.h
    return {"rel_fro": float(np.linalg.norm(d) / np.linalg.norm(ref.h)), "max_abs": float(np.abs(d).max()),
            "resid_f_of_gpu_H_by_oracle": O.residual_f(A, H), "oracle_resid_f": ref.resid_f,
            "oracle_sweeps": ref.sweeps, "oracle_ns_steps": ref.ns_steps, "oracle_status": ref.status}


# ------------------------------------------------------------ headline c2 --

def measure_c2(args, ibmi, lib, world, rank, local):
    import ctypes as C
    import numpy as np
    import torch
    import workloads as wl

    A = wl.c2_matern(P, seed=2)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    prec = ibmi.IBMI_MIXED if args.precision == "mixed" else ibmi.IBMI_FP64
    kw = dict(tol=TOL, max_sweeps=500, precision=prec, check_every=1)
    if prec == ibmi.IBMI_MIXED:
        kw.update(ns_theta=THETA, ns_max=8)
    plan = ibmi.ibmi_plan(P, K=K_SETS, h=H_OV, **kw)
    stream = torch.cuda.current_stream()

    def step():
        s, res = ibmi.ibmi_invert(plan, dA, dH, stream=stream)
        if s != ibmi.IBMI_OK:
            raise RuntimeError(f"inversion failed: {ibmi.ibmi_status_string(s)} {res}")
        return res

    for _ in range(max(3, args.warmup)):
        res = step()
    torch.cuda.synchronize()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks = ClockSampler(local).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = lib.ibmi_launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = lib.ibmi_launch_count() - launches0
    clk = clocks.stop()
    H_gpu = dH.cpu().numpy()
    # Kernel classes for the roofline: the same steps again with the library's
    # per-class CUDA events (they cost ~9% of a step and keep consecutive GEMMs
    # from overlapping, so the headline time above is taken without them).
    lib.ibmi_prof_enable(1)
    prof_steps = min(args.steps, 10)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    prof = {}
    for kc, name in enumerate(CLASSES):
        n, t, f, a = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        lib.ibmi_prof_get(kc, C.byref(n), C.byref(t), C.byref(f))
        lib.ibmi_prof_get_alg(kc, C.byref(a))
        prof[name] = (n.value, t.value, f.value, a.value)
    lib.ibmi_prof_enable(0)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * args.steps / (ms / 1000.0)
    last = results[-1]
    assert last["resid_f"] <= TOL, last

    # roofline of the dominant kernel class (by summed event time)
    peaks = measured_peaks()
    tensor_classes = set() if prec == ibmi.IBMI_FP64 else {"sweep_x", "sweep_s", "residual", "newton_schulz",
                                                          "invariants_tc"}
    dom = max((c for c in CLASSES if c != "other"), key=lambda c: prof[c][1])
    n_d, ms_d, fl_d, alg_d = prof[dom]
    achieved = (fl_d / n_d) / (ms_d / n_d / 1000.0) / 1e12 if n_d else None
    achieved_alg = alg_d / (ms_d / 1000.0) / 1e12 if ms_d else None
    if dom in tensor_classes:
        bound, peak, psrc = "tensor", peaks["bf16_sustained"], f"bf16 dense sustained ({peaks['src']})"
        kdesc = {"residual": "a6/a7 FP64-accurate residual: digit-pair BF16 GEMMs (tcgen05, exact FP32 accumulation)",
                 "newton_schulz": "a7 Newton-Schulz update: digit-pair BF16 GEMMs (tcgen05)",
                 "sweep_x": "a3 sweep product X = -W T (tcgen05 BF16x3)",
                 "sweep_s": "a4 sweep product X W^T (tcgen05 BF16x3)",
                 "invariants_tc": "a2 W = A_I^-1 A_I,: (tcgen05 digit pairs)"}[dom]
    else:
        bound, peak, psrc = "alu", FP64_PEAK_TFLOPS, "GB300 FP64 DFMA 1.25 TFLOP/s (nominal; no FP64 entry in measured peaks)"
        kdesc = {"sweep_x": "a3 sweep product X = -W T (FP64 DFMA)", "sweep_s": "a4 sweep product (FP64 DFMA)",
                 "residual": "a6 residual (FP64 DFMA)", "newton_schulz": "a7 Newton-Schulz (FP64 DFMA)",
                 "invariants": "a2 Cholesky + triangular solves (FP64 DFMA)"}.get(dom, dom)
    total_kernel_ms = sum(v[1] for v in prof.values())
    traffic, traffic_src = None, None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        ent = json.load(open(tpath)).get(f"{args.precision}/{dom}")
        if ent:
            traffic, traffic_src = ent.get("bytes_per_launch"), ent.get("source")
    step_s = ms / args.steps / 1000.0
    roofline = {
        "bound": bound, "kernel": kdesc, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
        "frac": (achieved / peak) if achieved else None,
        "frac_basis": "executed tensor-pipe flops (every slice / digit-pair product) of the dominant class; the "
                      ">= 60% target for the block GEMMs applies to this fraction of the BF16 peak",
        "achieved_algorithmic": achieved_alg,
        "frac_algorithmic": (achieved_alg / peak) if achieved_alg else None,
        "frac_algorithmic_basis": "flops of the products the method asks for (2 p^3 per residual, its share "
                                  "for a residual that keeps part of its digit pairs) / class time / peak",
        "step_frac_algorithmic": last["flops"] / step_s / 1e12 / peak,
        "traffic": traffic, "traffic_source": traffic_src, "peak_source": psrc,
        "launches": n_d, "share_of_kernel_time": ms_d / total_kernel_ms if total_kernel_ms else None,
        "timing": f"per-class CUDA events on the launching stream over {prof_steps} further steps of the "
                  "same workload (instrumented pass; the headline time is uninstrumented)",
        "classes": {k: {"launches": v[0], "ms": round(v[1], 3),
                        "tflops": round(v[2] / (v[1] / 1000.0) / 1e12, 2) if v[1] > 0 else None,
                        "tflops_algorithmic": round(v[3] / (v[1] / 1000.0) / 1e12, 2) if v[1] > 0 else None}
                    for k, v in prof.items() if v[0]}}

    # end to end through the host-buffer entry point
    Ah = torch.from_numpy(A).pin_memory().numpy()
    Hh = torch.empty((P, P), dtype=torch.float64).pin_memory().numpy()
    s, r = ibmi.ibmi_invert_host(plan, Ah, Hh, stream=stream)
    assert s == ibmi.IBMI_OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, r = ibmi.ibmi_invert_host(plan, Ah, Hh, stream=stream)
        assert s == ibmi.IBMI_OK
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * args.steps / e2e_s, "unit": "inverses/s",
           "h2d_bytes_per_step": int(A.nbytes), "d2h_bytes_per_step": int(A.nbytes)}

    fp64_cmp = None
    if prec == ibmi.IBMI_MIXED and not args.no_fp64_compare:
        plan64 = ibmi.ibmi_plan(P, K=K_SETS, h=H_OV, tol=TOL, max_sweeps=500, precision=ibmi.IBMI_FP64,
                                check_every=1)
        dH64 = torch.empty_like(dA)
        s64, r64 = ibmi.ibmi_invert(plan64, dA, dH64, stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64, r64 = ibmi.ibmi_invert(plan64, dA, dH64, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_cmp = {"value": 1000.0 / f0.elapsed_time(f1), "unit": "inverses/s", "status": s64,
                    "sweeps": r64["sweeps"], "resid_f": r64["resid_f"], "steps": 1,
                    "note": "plain FP64 (DFMA) IBMI on the same GPU, same tolerance"}
        plan64.close()
        del dH64

    cpu, err = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        secs, ref = oracle_solve(A, K_SETS, H_OV)
        cpu = {"value": 1.0 / secs, "unit": "inverses/s", "cores": host_cores(), "kind": "oracle",
               "sample": f"one complete oracle solve of the same workload ({ref.sweeps} sweeps + "
                         f"{ref.ns_steps} Newton-Schulz steps, {secs:.1f} s, status {ref.status})"}
        err = vs_oracle(A, H_gpu, ref)
    plan.close()
    line = {"metric": METRIC, "value": value, "unit": "inverses/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == ibmi.IBMI_FP64 else "bf16 (tcgen05 split/digit-sliced) + f64",
            "data": "synthetic",
            "config": {"workload": "matern32_p4096_K8_h32", "p": P, "K": K_SETS, "h": H_OV,
                       "tol": TOL, "precision": args.precision, "ns_theta": THETA if prec == ibmi.IBMI_MIXED else 0,
                       "sweeps": last["sweeps"], "ns_steps": last["ns_steps"], "resid_f": last["resid_f"],
                       "l2": "inputs larger than L2 (A, H 134 MB each); no flush",
                       "parallelism": f"replicas{world}"},
            "achieved_tflops_step": last["flops"] / step_s / 1e12,
            "vs_oracle": err, "roofline": roofline, "fp64_gpu": fp64_cmp, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk}
    return line


# --------------------------------------------------------------------- c3 --

def measure_c3(ibmi, lib, local, steps=2):
    """p = 8192 random SPD, K = 2, h = 1024, mixed precision to 1e-10, from
    the initial approximation T_0 = A_{I_1^c}^{-1} (Section 5.6; 66 sweeps
    against 257 from the identity, whose solve is timed once beside it)."""
    import torch
    import workloads as wl
    p, K, h = 8192, 2, 1024
    A = wl.c3_random_spd(p, seed=3)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    del A
    stream = torch.cuda.current_stream()
    plan = ibmi.ibmi_plan(p, K=K, h=h, tol=TOL, max_sweeps=500, precision=ibmi.IBMI_MIXED, ns_theta=THETA, ns_max=8,
                          init=ibmi.IBMI_INIT_SCHUR)
    s, r = ibmi.ibmi_invert(plan, dA, dH, stream=stream)   # warm-up (captures nothing; plan pools exist)
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = lib.ibmi_launch_count()
    e0.record(stream)
    res = []
    for _ in range(steps):
        s, r = ibmi.ibmi_invert(plan, dA, dH, stream=stream)
        res.append((s, r))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    clk = clocks.stop()
    launches = lib.ibmi_launch_count() - l0
    s, r = res[-1]
    # one more solve with the library's per-class events: the tensor-pipe
    # rate of the sweep products at these shapes (5120-row sets fill the GPU)
    import ctypes as C
    lib.ibmi_prof_enable(1)
    ibmi.ibmi_invert(plan, dA, dH, stream=stream)
    torch.cuda.synchronize()
    peak = measured_peaks()["bf16_sustained"]
    classes = {}
    for kc, name in enumerate(CLASSES):
        n, t, f, a = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
        lib.ibmi_prof_get(kc, C.byref(n), C.byref(t), C.byref(f))
        lib.ibmi_prof_get_alg(kc, C.byref(a))
        if n.value == 0:
            continue
        tf = f.value / (t.value / 1000.0) / 1e12 if t.value > 0 else 0.0
        classes[name] = {"launches": n.value, "ms": round(t.value, 3), "tflops": round(tf, 2),
                         "tflops_algorithmic": round(a.value / (t.value / 1000.0) / 1e12, 2) if t.value > 0 else 0.0}
        if name in ("sweep_x", "sweep_s", "residual", "newton_schulz", "invariants_tc"):
            classes[name]["frac_of_bf16_sustained"] = round(tf / peak, 3)
    lib.ibmi_prof_enable(0)
    plan.close()
    # the same solve from the identity (the paper's default start), once
    ident = None
    try:
        pl = ibmi.ibmi_plan(p, K=K, h=h, tol=TOL, max_sweeps=500, precision=ibmi.IBMI_MIXED, ns_theta=THETA, ns_max=8)
        ibmi.ibmi_invert(pl, dA, dH, stream=stream)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        si, ri = ibmi.ibmi_invert(pl, dA, dH, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        ident = {"ms_per_inverse": f0.elapsed_time(f1), "status": si, "sweeps": ri["sweeps"],
                 "ns_steps": ri["ns_steps"], "resid_f": ri["resid_f"]}
        pl.close()
    except Exception as e:   # reported, not fatal
        ident = {"error": str(e)}
    # plain FP64 IBMI on the same matrix: the time of one FP64 sweep (two runs
    # that differ by two sweeps and have the same single stop test)
    fp64 = None
    try:
        t = []
        for ms_cap in (1, 3):
            pl = ibmi.ibmi_plan(p, K=K, h=h, tol=0.0, max_sweeps=ms_cap, check_every=ms_cap, precision=ibmi.IBMI_FP64)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            ibmi.ibmi_invert(pl, dA, dH, stream=stream)
            f1.record(stream)
            torch.cuda.synchronize()
            t.append(f0.elapsed_time(f1))
            pl.close()
        fp64 = {"sweep_ms": (t[1] - t[0]) / 2.0, "plan_plus_one_sweep_and_residual_ms": t[0],
                "note": "plain FP64 (DFMA) IBMI on the same GPU: time of one sweep; its converged solve "
                        "needs hundreds of sweeps on this matrix (the mixed path's sweeps alone are shown)"}
    except Exception as e:   # reported, not fatal
        fp64 = {"error": str(e)}
    return {"workload": "random_spd_p8192_K2_h1024_init_schur", "metric": "SPD inverses/s @ rho_F<=1e-10",
            "value": 1000.0 / ms, "unit": "inverses/s", "ms_per_inverse": ms, "steps": steps, "warmup": 1,
            "status": s, "sweeps": r["sweeps"], "ns_steps": r["ns_steps"], "resid_f": r["resid_f"],
            "achieved_tflops_algorithmic": r["flops"] / (ms / 1000.0) / 1e12,
            "gpu_launches_per_inverse": launches / steps, "classes_instrumented": classes,
            "identity_start": ident, "fp64_gpu": fp64, "clocks": clk,
            "dtype": "bf16 (tcgen05 split/digit-sliced) + f64"}


# --------------------------------------------------------------------- c4 --

def measure_c4(ibmi, lib, local, args, steps=3):
    """512 squared-exponential covariance matrices on seeded 3-D points, p in
    {64, ..., 1024}, one ibmi_invert_batched call per step (mixed precision);
    plus mixed vs FP64 on a 64-matrix sample and the oracle on 8 of them."""
    import numpy as np
    import torch
    import workloads as wl
    mats = wl.c4_batch(n=args.batch_n, seed=4)
    As = [torch.from_numpy(A).cuda() for A in mats]
    Hs = [torch.empty_like(a) for a in As]
    for _ in range(2):   # the first call also tunes (K, h) per size bucket
        ibmi.ibmi_invert_batched(As, Hs, precision=ibmi.IBMI_MIXED, workers=16)
    torch.cuda.synchronize()
    clocks = ClockSampler(local).start()
    l0 = lib.ibmi_launch_count()
    t0 = time.perf_counter()
    for _ in range(steps):
        s, res = ibmi.ibmi_invert_batched(As, Hs, precision=ibmi.IBMI_MIXED, workers=16)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    clk = clocks.stop()
    launches = (lib.ibmi_launch_count() - l0) / steps
    bstats = ibmi.ibmi_batch_last_stats()
    ok = sum(r["status"] == 0 for r in res)
    rf = sorted(r["resid_f"] for r in res)
    flops = sum(r["flops"] for r in res)
    # like for like: the same 64 matrices, mixed and plain FP64 batched
    rng = np.random.default_rng(44)
    sel = sorted(rng.choice(len(mats), 64, replace=False).tolist())
    sA, sH = [As[i] for i in sel], [Hs[i] for i in sel]
    out = {}
    first_of_size = {}
    for k, i in enumerate(sel):
        first_of_size.setdefault(mats[i].shape[0], k)
    warm = sorted(first_of_size.values())
    for name, prec, tune in (("mixed", ibmi.IBMI_MIXED, 1), ("fp64", ibmi.IBMI_FP64, 0)):
        # plans for every size of the sample (FP64: default partitions, no tuning runs)
        ibmi.ibmi_invert_batched([sA[k] for k in warm], [sH[k] for k in warm], precision=prec, workers=16,
                                 autotune=tune)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s2, r2 = ibmi.ibmi_invert_batched(sA, sH, precision=prec, workers=16, autotune=tune)
        torch.cuda.synchronize()
        d2 = time.perf_counter() - t1
        out[name] = {"value": len(sel) / d2, "unit": "inverses/s", "seconds": d2,
                     "converged": sum(r["status"] == 0 for r in r2),
                     "resid_f_max": max(r["resid_f"] for r in r2)}
    # oracle on 8 of them (the CPU reference for this workload)
    from oracle import ibmi_oracle as O
    t2 = time.perf_counter()
    for i in sel[:8]:
        p = mats[i].shape[0]
        K = 2 if p <= 256 else 3
        O.ibmi(mats[i], O.partition(p, K, max(4, round(0.1 * (p // K)))), tol=TOL, max_sweeps=300, ns_theta=0.5)
    cpu_s = time.perf_counter() - t2
    ibmi.ibmi_batch_release()
    return {"workload": "se3d_batch512", "metric": "SPD inverses/s, batch of 512 squared-exponential matrices "
                                                  "p in 64..1024, rho_F<=1e-10",
            "value": len(mats) / dt, "unit": "inverses/s", "ms_per_batch": dt * 1000.0, "steps": steps,
            "warmup": 2, "converged": ok, "not_converged": len(res) - ok, "resid_f_median": rf[len(rf) // 2],
            "resid_f_max": rf[-1], "achieved_tflops_algorithmic": flops / dt / 1e12,
            "gpu_launches_per_batch": launches, "batch_stats": bstats, "sample64": out,
            "mixed_over_fp64_on_sample": out["mixed"]["value"] / out["fp64"]["value"],
            "cpu_oracle_sample": {"value": 8.0 / cpu_s, "unit": "inverses/s", "matrices": 8,
                                  "cores": host_cores(), "kind": "oracle"},
            "clocks": clk, "dtype": "bf16 (tcgen05 split/digit-sliced) + f64", "workers": 16}


# --------------------------------------------------------------------- c5 --

def _drain(srv, ibmi, sub):
    status = {}
    for rid, p in sub:
        while True:
            st, _, _ = srv.poll(rid, p)
            if st != ibmi.IBMI_NOT_READY:
                status[st] = status.get(st, 0) + 1
                break
            time.sleep(0.001)
    return status


def serve_trace(srv, ibmi, trace, pool, seconds):
    srv.reset_stats()
    t0 = time.perf_counter()
    sub = []
    for i, r in enumerate(trace):
        if r.t_arrival > seconds:
            break
        now = time.perf_counter() - t0
        if r.t_arrival > now:
            time.sleep(r.t_arrival - now)
        A = pool[i % len(pool)]
        sub.append((srv.submit(A), A.shape[0]))
    t_sub = time.perf_counter() - t0
    status = _drain(srv, ibmi, sub)
    t_all = time.perf_counter() - t0
    st = srv.stats()
    return {"submitted": len(sub), "submit_window_s": t_sub, "drain_s": t_all - t_sub,
            "drained_inverses_per_s": len(sub) / t_all, "p50_s": st["p50_s"], "p99_s": st["p99_s"],
            "status_counts": {str(k): v for k, v in status.items()}}


def measure_c5(ibmi, local, args):
    """Poisson arrivals of inversion requests (p log-uniform in [128, 4096];
    KMS, Matern-3/2 and compound-symmetry families in equal parts) into the
    continuous-batching server with a 64 GB budget, at each offered rate.
    Matrices are drawn from a pool of 48 pre-generated requests of the trace
    (generation is host work)."""
    import workloads as wl
    rates = [float(x) for x in args.serve_rates.split(",") if x]
    base = wl.c5_trace(3.0, rate=2000.0, seed=5)
    pool = [r.matrix(seed=100 + i) for i, r in enumerate(base[:48])]
    srv = ibmi.Server(64 << 30, workers=16)
    for _ in range(2):   # every pool entry served twice: each worker holds the plans of its sizes
        ids = [(srv.submit(A), A.shape[0]) for A in pool]
        _drain(srv, ibmi, ids)
    runs = []
    clocks = ClockSampler(local).start()
    for rate in rates:
        seconds = args.serve_seconds if rate >= 1000 else max(args.serve_seconds, 48.0 / rate)
        trace = wl.c5_trace(seconds + 1.0, rate=rate, seed=5)
        r = serve_trace(srv, ibmi, trace, pool, seconds)
        r.update({"offered_rate": rate, "trace_seconds": seconds})
        runs.append(r)
    clk = clocks.stop()
    srv.close()
    # plain FP64 served on a sample of the same requests (orders <= 1024: an
    # FP64 compound-symmetry request of order 4096 alone runs for minutes),
    # the mixed server on the same sample beside it
    sample = [A for A in pool if A.shape[0] <= 1024][:8]
    fp = {}
    for name, prec in (("mixed", ibmi.IBMI_MIXED), ("fp64", ibmi.IBMI_FP64)):
        s2 = ibmi.Server(64 << 30, workers=16, precision=prec)
        t0 = time.perf_counter()
        ids = [(s2.submit(A), A.shape[0]) for A in sample]
        status = _drain(s2, ibmi, ids)
        dt = time.perf_counter() - t0
        s2.close()
        fp[name] = {"value": len(sample) / dt, "unit": "inverses/s", "seconds": dt,
                    "status_counts": {str(k): v for k, v in status.items()}}
    return {"workload": "serve_poisson", "metric": "served SPD inverses/s and p50/p99 latency",
            "unit": "inverses/s", "value": runs[0]["drained_inverses_per_s"], "rates": runs,
            "budget_gb": 64, "workers": 16, "pool": len(pool),
            "sample8_cold": fp, "clocks": clk,
            "note": "sample8_cold: 8 requests of order <= 1024 from the pool on a fresh server each "
                    "(plan creation included), mixed vs plain FP64"}


# -------------------------------------------------------------- reference --

def reference_arm(args):
    import workloads as wl
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    A = wl.c2_matern(P, seed=2)
    for _ in range(args.warmup):
        oracle_solve(A, K_SETS, H_OV)
    times, ref = [], None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, ref = oracle_solve(A, K_SETS, H_OV)
        times.append(s)
    elapsed = time.perf_counter() - t0
    value = args.steps / elapsed
    desc = (f"one complete oracle solve per step ({ref.sweeps} sweeps + {ref.ns_steps} Newton-Schulz steps, "
            f"status {ref.status}, median {statistics.median(times):.2f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "inverses/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "matern32_p4096_K8_h32", "p": P, "K": K_SETS, "h": H_OV,
                       "tol": TOL, "ns_theta": THETA},
            "cpu_baseline": {"value": value, "unit": "inverses/s", "cores": host_cores(),
                             "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": "inverses/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- main --

def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as ibmi
    from paper_2502_06377_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload in ("c3", "batch", "serve"):
        if rank == 0:
            fn = {"c3": lambda: measure_c3(ibmi, lib, local), "batch": lambda: measure_c4(ibmi, lib, local, args),
                  "serve": lambda: measure_c5(ibmi, local, args)}[args.workload]
            print(json.dumps(fn()), flush=True)
        return 0
    line = measure_c2(args, ibmi, lib, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return 0
    if args.workload == "all" and world == 1:
        configs = {}
        for name, fn in (("c3", lambda: measure_c3(ibmi, lib, local)),
                         ("c4", lambda: measure_c4(ibmi, lib, local, args)),
                         ("c5", lambda: measure_c5(ibmi, local, args))):
            t0 = time.perf_counter()
            try:
                configs[name] = fn()
            except Exception as e:   # a failing sub-measurement is reported, the headline stands
                configs[name] = {"error": f"{type(e).__name__}: {e}"}
            configs[name]["wall_s"] = time.perf_counter() - t0
            torch.cuda.synchronize()
        line["configs"] = configs
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
