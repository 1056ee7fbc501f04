#!/usr/bin/env python
"""IBMI inversion benchmark on GB300.

Metric: SPD inverses per second at ||I - A H||_F / sqrt(p) <= 1e-10, on the
p = 4096 Matern-3/2 workload (4096 seeded points in the unit square sorted by
x, length scale 0.1, unit variance, nugget 1e-2; K = 8 sets of 544/576 rows
with 64-row overlap).  One step = one complete inversion through the C ABI
(block invariants, sweeps, stop tests, optional Newton-Schulz tail), with A
resident in HBM.  A and H are 134 MB each, larger than the 129 MB L2, so no
L2 flush is needed between steps.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (block invariants + one sweep + one residual, scaled to a full solve
by the sweep count the GPU path needs) on the host cores.

Multi-GPU: every rank inverts its own copy (independent problems, no
collective); value = inverses of all ranks / max-over-ranks time.
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
P, K_SETS, H_OV, TOL = 4096, 8, 32, 1e-10
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
    ap.add_argument("--workload", default="c2", choices=["c2", "batch", "serve"],
                    help="c2: the headline single-matrix line; batch: 512 squared-exponential "
                         "matrices of uneven order; serve: Poisson request trace")
    ap.add_argument("--batch-n", type=int, default=512)
    ap.add_argument("--serve-seconds", type=float, default=0.25)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
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
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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


# ----------------------------------------------------------- cpu baseline --

def oracle_sample(A, sweeps: int, checks: int, ns_steps: int = 0):
    """Times the oracle on the block invariants, one sweep, one residual and
    (if ns_steps) one Newton-Schulz step of the workload, and scales to a full
    solve of `sweeps` sweeps, `checks` stop tests and `ns_steps` Newton-Schulz
    steps (each followed by a residual).  Returns (inverses/s, seconds of CPU
    work actually spent, description)."""
    from oracle import ibmi_oracle as O
    import numpy as np
    sets = O.partition(P, K_SETS, H_OV)
    t0 = time.perf_counter()
    invs = [O.block_invariants(A, lo, hi) for lo, hi in sets]
    t1 = time.perf_counter()
    H = np.eye(P)
    for inv in invs:
        O.block_update(H, inv)
    t2 = time.perf_counter()
    O.residual_f(A, H)
    t3 = time.perf_counter()
    t_ns = 0.0
    if ns_steps:
        O.newton_schulz_step(A, H)
        t_ns = time.perf_counter() - t3
    spent = time.perf_counter() - t0
    full = (t1 - t0) + sweeps * (t2 - t1) + (checks + ns_steps) * (t3 - t2) + ns_steps * t_ns
    desc = (f"oracle block invariants of all {K_SETS} sets + 1 sweep + 1 residual"
            + (" + 1 Newton-Schulz step" if ns_steps else "")
            + f" ({spent:.1f} s), scaled to {sweeps} sweeps, {checks} residual checks"
            + (f" and {ns_steps} Newton-Schulz steps" if ns_steps else ""))
    return 1.0 / full, spent, desc


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# -------------------------------------------------------------------- main --

def run_batch(args):
    """512 squared-exponential covariance matrices on seeded 3-D points, p in
    {64, ..., 1024}, one ibmi_invert_batched call per step."""
    import numpy as np
    import torch
    import workloads as wl
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as ibmi
    from paper_2502_06377_gb300 import shard
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    all_mats = wl.c4_batch(n=args.batch_n, seed=4)
    mine = shard.shard_by_cost([A.shape[0] for A in all_mats], world, rank)   # no data-path collective
    mats = [all_mats[i] for i in mine]
    As = [torch.from_numpy(A).cuda() for A in mats]
    Hs = [torch.empty_like(a) for a in As]
    prec = ibmi.IBMI_MIXED if args.precision == "mixed" else ibmi.IBMI_FP64
    for _ in range(max(1, args.warmup)):          # the first call also tunes (K, h) per size
        ibmi.ibmi_invert_batched(As, Hs, precision=prec, workers=16)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    lib = ibmi._lib.load()
    l0 = lib.ibmi_launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s, res = ibmi.ibmi_invert_batched(As, Hs, precision=prec, workers=16)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    dt = shard.max_over_ranks((time.perf_counter() - t0) / args.steps, device="cuda")
    launches = lib.ibmi_launch_count() - l0
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    ok = sum(r["status"] == 0 for r in res)
    flops = sum(r["flops"] for r in res)
    rf = sorted(r["resid_f"] for r in res)
    line = {"metric": "SPD inverses/s, batch of 512 squared-exponential matrices p in 64..1024",
            "value": len(all_mats) / dt, "unit": "inverses/s", "n_gpus": world, "steps": args.steps,
            "scaling": "strong (the batch is split across ranks by estimated cost)",
            "warmup": args.warmup, "ms_per_step": dt * 1000, "higher_is_better": True,
            "dtype": "bf16 (tcgen05) + f64" if prec == ibmi.IBMI_MIXED else "f64", "data": "synthetic",
            "config": {"workload": "se3d_batch512", "precision": args.precision, "workers": 16,
                       "note": "rank 0's share shown for convergence counts"},
            "converged": ok, "not_converged": len(res) - ok,
            "resid_f_median": rf[len(rf) // 2], "resid_f_max": rf[-1],
            "achieved_tflops": flops / dt / 1e12, "gpu_launches": launches,
            "sum_p3": float(sum(float(m.shape[0]) ** 3 for m in mats))}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Poisson arrivals of inversion requests (p log-uniform in [128, 4096];
    KMS, Matern-3/2 and compound-symmetry families in equal parts) into the
    continuous-batching server with a 64 GB budget.  Matrices are drawn from a
    pool of 48 pre-generated requests of the trace (generation is host work)."""
    import numpy as np
    import workloads as wl
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as ibmi
    trace = wl.c5_trace(args.serve_seconds + 2.0, rate=args.serve_rate, seed=5)
    pool_reqs = trace[:48]
    pool = [r.matrix(seed=100 + i) for i, r in enumerate(pool_reqs)]
    srv = ibmi.Server(64 << 30, workers=16)
    # warm-up on the same server: every pool entry a few times, so that each
    # worker holds the plans (and captured graphs) of the sizes it serves
    for _ in range(max(1, args.warmup)):
        ids = [(srv.submit(A), A.shape[0]) for A in pool]
        for rid, p in ids:
            while srv.poll(rid, p)[0] == ibmi.IBMI_NOT_READY:
                time.sleep(0.001)
    srv.reset_stats()
    t0 = time.perf_counter()
    sub = []
    for i, r in enumerate(trace):
        now = time.perf_counter() - t0
        if r.t_arrival > now:
            time.sleep(r.t_arrival - now)
        if r.t_arrival > args.serve_seconds:
            break
        A = pool[i % len(pool)]
        sub.append((srv.submit(A), A.shape[0]))
    t_sub = time.perf_counter() - t0
    status = {}
    for rid, p in sub:
        while True:
            st, _, _ = srv.poll(rid, p)
            if st != ibmi.IBMI_NOT_READY:
                status[st] = status.get(st, 0) + 1
                break
            time.sleep(0.001)
    t_all = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    line = {"metric": "served SPD inverses/s and latency (Poisson trace)", "value": len(sub) / t_all,
            "unit": "inverses/s", "p50_s": stats["p50_s"], "p99_s": stats["p99_s"],
            "offered_rate": args.serve_rate, "submitted": len(sub), "submit_window_s": t_sub,
            "drain_s": t_all - t_sub, "status_counts": {str(k): v for k, v in status.items()},
            "config": {"workload": "serve_poisson", "budget_gb": 64, "workers": 16,
                       "pool": len(pool), "seconds": args.serve_seconds}, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "ours" and args.workload == "batch":
        return run_batch(args)
    if args.impl == "ours" and args.workload == "serve":
        return run_serve(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import numpy as np
    import workloads as wl

    if args.impl == "reference":
        if rank != 0:
            return 0
        A = wl.c2_matern(P, seed=2)
        # the oracle's own hybrid solve of this workload (sweeps until
        # ||I - AH||_F <= 0.5, then Newton-Schulz) takes 5 sweeps and 3 steps
        sweeps, checks, ns = 5, 5, 3
        for _ in range(args.warmup):
            oracle_sample(A, sweeps, checks, ns)
        vals, spent, desc = [], 0.0, ""
        t0 = time.perf_counter()
        for _ in range(args.steps):
            v, s, desc = oracle_sample(A, sweeps, checks, ns)
            vals.append(v)
            spent += s
        elapsed = time.perf_counter() - t0
        value = statistics.median(vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "inverses/s",
                "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * elapsed / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "matern32_p4096_K8_h32", "p": P, "K": K_SETS, "h": H_OV,
                           "tol": TOL},
                "cpu_baseline": {"value": value, "unit": "inverses/s", "cores": host_cores(),
                                 "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": "inverses/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2502_06377_gb300 as ibmi
    from paper_2502_06377_gb300 import _lib
    lib = _lib.load()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    A = wl.c2_matern(P, seed=2)
    dA = torch.from_numpy(A).cuda()
    dH = torch.empty_like(dA)
    prec = ibmi.IBMI_MIXED if args.precision == "mixed" else ibmi.IBMI_FP64
    kw = dict(tol=TOL, max_sweeps=500, precision=prec)
    if prec == ibmi.IBMI_MIXED:
        kw.update(ns_theta=0.9, ns_max=8, check_every=1)
    else:
        kw.update(check_every=1)
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
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = lib.ibmi_launch_count()
    torch.cuda.synchronize()
    e0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(step())
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = lib.ibmi_launch_count() - launches0
    clk = clocks.stop()
    # Kernel classes for the roofline: the same steps again with the library's
    # per-class CUDA events (they cost ~9% of a step and keep consecutive GEMMs
    # from overlapping, so the headline time above is taken without them).
    import ctypes as C
    lib.ibmi_prof_enable(1)
    prof_steps = min(args.steps, 10)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    prof = {}
    for kc, name in enumerate(CLASSES):
        n, t, f = C.c_int64(), C.c_double(), C.c_double()
        lib.ibmi_prof_get(kc, C.byref(n), C.byref(t), C.byref(f))
        prof[name] = (n.value, t.value, f.value)
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
    n_d, ms_d, fl_d = prof[dom]
    achieved = (fl_d / n_d) / (ms_d / n_d / 1000.0) / 1e12 if n_d else None
    if dom in tensor_classes:
        bound, peak, psrc = "tensor", peaks["bf16_sustained"], f"bf16 dense sustained ({peaks['src']})"
        kdesc = {"residual": "a6/a7 FP64-accurate residual: digit-pair BF16 GEMMs (tcgen05, exact FP32 accumulation)",
                 "newton_schulz": "a7 Newton-Schulz update: digit-pair BF16 GEMMs (tcgen05)",
                 "sweep_x": "a3 sweep product X = -W T (tcgen05 BF16x3)",
                 "sweep_s": "a4 sweep product X W^T (tcgen05 BF16x3)",
                 "invariants_tc": "a2 W = A_I^-1 A_I,: (tcgen05 BF16x3)"}[dom]
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
    roofline = {"bound": bound, "kernel": kdesc, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic, "traffic_source": traffic_src,
                "peak_source": psrc,
                "launches": n_d, "share_of_kernel_time": ms_d / total_kernel_ms if total_kernel_ms else None,
                "timing": f"per-class CUDA events on the launching stream over {prof_steps} further steps of the "
                          "same workload (instrumented pass; the headline time is uninstrumented)",
                "classes": {k: {"launches": v[0], "ms": round(v[1], 3),
                                "tflops": round(v[2] / (v[1] / 1000.0) / 1e12, 2) if v[1] > 0 else None}
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
        s64, r64 = ibmi.ibmi_invert(plan64, dA, dH, stream=stream)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        s64, r64 = ibmi.ibmi_invert(plan64, dA, dH, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize()
        fp64_cmp = {"value": 1000.0 / f0.elapsed_time(f1), "unit": "inverses/s", "status": s64,
                    "sweeps": r64["sweeps"], "resid_f": r64["resid_f"], "steps": 1,
                    "note": "plain FP64 (DFMA) IBMI on the same GPU, same tolerance"}
        plan64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, spent, desc = oracle_sample(A, last["sweeps"], last["sweeps"], last["ns_steps"])
        cpu = {"value": v, "unit": "inverses/s", "cores": host_cores(), "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "inverses/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == ibmi.IBMI_FP64 else "bf16 (tcgen05 split/digit-sliced) + f64",
                "data": "synthetic",
                "config": {"workload": "matern32_p4096_K8_h32", "p": P, "K": K_SETS, "h": H_OV,
                           "tol": TOL, "precision": args.precision, "sweeps": last["sweeps"],
                           "ns_steps": last["ns_steps"], "resid_f": last["resid_f"],
                           "l2": "inputs larger than L2 (A, H 134 MB each); no flush",
                           "parallelism": f"replicas{world}"},
                "achieved_tflops_step": last["flops"] / (ms / args.steps / 1000.0) / 1e12,
                "roofline": roofline, "fp64_gpu": fp64_cmp, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
