#!/usr/bin/env python3
"""Benchmark of the DMRG operator rotation O'_k = U^T (O_k (x) I_d) U on GB300.

Workload (one "step" = one rotation of the whole operator batch): the dense
Hubbard-shaped step d = 4, m = 400 -> m*d = 1600 -> m' = 400, K = 150
operators per GPU (50 sites x {n_up-like, two dense}), seeded synthetic
inputs resident in HBM, L2 flushed (512 MiB write) between timed steps.
The headline precision is BF16x3; TF32 and the plain FP64 GPU path are timed
on the same inputs and reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun each rank rotates its uniform-matrix-distribution slice of
K*N operators (no collective on the data path); value = all operators / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rotated operators/s and eff. TFLOP/s (BF16×3, TF32 vs FP64 path) at m=400,K=150"
UNIT = "rotated operators/s"
WORKLOAD = "dense_m400_k150"
D, M, MP, K_PER_GPU = 4, 400, 400, 150
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic.json")
KERNEL_SOURCES = ["paper_0909_5662_gb300/csrc/tc.cu", "paper_0909_5662_gb300/csrc/tc_pair.cu",
                  "paper_0909_5662_gb300/csrc/tc_common.cuh", "paper_0909_5662_gb300/csrc/ptx.cuh",
                  "paper_0909_5662_gb300/csrc/internal.h"]


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, which):
        """Brackets the timed region: samples outside it are dropped."""
        setattr(self, which, time.monotonic())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = getattr(self, "t_begin", -1e30)
        t1 = getattr(self, "t_end", 1e30)
        inside = [ln for t, ln in self.lines if t0 <= t <= t1]
        for ln in inside:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "samples taken during the timed BF16x3 steps",
                "power_w_median": statistics.median(power) if power else None,
                "power_w_max": max(power) if power else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def traffic_for(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or None
    if absent or taken on a different version of the kernel sources."""
    try:
        with open(TRAFFIC_FILE) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return None
    if data.get("source_hash") != kernel_source_hash():
        return None
    ent = data.get("kernels", {}).get(kernel)
    return None if ent is None else ent.get("bytes_per_launch")


# ---------------------------------------------------------------------------- CPU oracle leg
def cpu_oracle_sample(w, budget_s: float = 12.0, max_ops: int = 150):
    """The FP64 CPU oracle as it stands, on host cores, on a bounded sample of the
    same workload: operators 0.. of the batch until about budget_s of work."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    n = min(max_ops, max(cores, 8))
    t0 = time.perf_counter()
    oracle.rotate_dense(w.U, w.O[:n], w.d)
    dt = time.perf_counter() - t0
    done, total_t = n, dt
    while total_t < budget_s and done < 4 * max_ops:
        n2 = min(max_ops, max(cores, int(n * max(1.0, (budget_s - total_t) / max(dt, 1e-3)))))
        t0 = time.perf_counter()
        oracle.rotate_dense(w.U, w.O[:n2], w.d)
        dt = time.perf_counter() - t0
        done += n2
        total_t += dt
        n = n2
    return {"value": done / total_t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d rotations of the first operators of %s (FP64 loops, UMD split over "
                      "%d OpenMP threads), %.1f s" % (done, WORKLOAD, cores, total_t)}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, on the host cores.  Each
    step rotates a bounded sample of the workload's operators (the first n of the
    batch, n chosen from the warm-up steps so that the timed steps take about 90 s in
    all, at least one operator and at most the whole batch); value = operators rotated
    in the timed steps / their total time, and ms_per_step is the measured time of one
    such step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from workloads import dense_config
    oracle.build()
    w = dense_config(WORKLOAD)
    cores = oracle.num_threads()
    n = min(K_PER_GPU, cores)
    rate = None
    for _ in range(args.warmup):
        t0 = time.perf_counter()
        oracle.rotate_dense(w.U, w.O[:n], w.d)
        rate = n / (time.perf_counter() - t0)
    budget_s = 90.0
    n = int(max(1, min(K_PER_GPU, rate * budget_s / max(args.steps, 1))))
    if cores <= n < K_PER_GPU:
        n = n // cores * cores   # whole rounds of the UMD split
    t_total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.rotate_dense(w.U, w.O[:n], w.d)
        t_total += time.perf_counter() - t0
    done = n * args.steps
    v = done / t_total
    res = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "each step rotates the first %d of the %d operators of %s (FP64 loops, UMD "
                     "split over %d OpenMP threads); %d timed steps, %.1f s" %
                     (n, K_PER_GPU, WORKLOAD, cores, args.steps, t_total)}
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "%s (d=4, m=400, m'=400, K=150)" % WORKLOAD,
                       "arm": "FP64 CPU oracle (the reference arm of this project)",
                       "operators_per_step": n},
            "cpu_baseline": res,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- GPU leg
# ---------------------------------------------------------------------------- blocked and adjoint reports
def _timed(fn, steps, warmup, flush):
    """Mean CUDA-event time (ms) of fn over `steps` calls after `warmup`, L2 flushed
    between calls (the flush itself is outside the timed intervals)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def blocked_report(steps, precisions, flush):
    """The U(1)xU(1) block-sparse rotation (grouped launches over the realised sector
    problems) on both synthetic sector laws: time per call for every precision,
    logical TFLOP/s over the realised problems, and the error of each reduced path
    against the FP64 GPU path on the same inputs."""
    import torch
    import paper_0909_5662_gb300 as P
    from workloads import blocked_config

    dev = flush.device
    res = {}
    for name in ("blocked_m1000_k200_s4", "blocked_m1000_k200_s1.2"):
        w = blocked_config(name)
        plan = P.dmrg_blocked_plan_create(w.block_sectors, w.site_shifts, w.kept_sectors, w.op_shifts)
        n1, n2, flops = plan.stats()
        Ub = torch.from_numpy(w.U_blocks).to(dev)
        O64 = torch.from_numpy(w.O_blocks).to(dev)
        O32 = O64.float()
        ref = P.dmrg_rotate_ops_blocked(plan, Ub, O64, "fp64")
        small = max(max(s[2] for s in w.block_sectors), max(s[2] for s in w.kept_sectors)) <= 32
        row = {"path": "fused small-sector kernel (FP32; FP64 for fp64)" if small else
                       "grouped GEMMs (tcgen05 for bf16x3/tf32, plain FMA for fp32/fp64)",
               "problems_first": n1, "problems_second": n2, "flops_per_call": flops,
               "sectors": len(w.block_sectors), "operators": w.K,
               "block_rows_max": max(s[2] for s in w.block_sectors)}
        for prec in precisions:
            O = O64 if prec == "fp64" else O32
            out = P.dmrg_rotate_ops_blocked(plan, Ub, O, prec)
            n = steps if prec != "fp64" else max(1, steps // 10)
            ms = _timed(lambda: P.dmrg_rotate_ops_blocked(plan, Ub, O, prec, out=out), n, 3, flush)
            kt = _with_kernel_timing(lambda: P.dmrg_rotate_ops_blocked(plan, Ub, O, prec, out=out),
                                     min(n, 20), flush)
            P.dmrg_sync_status()
            err = float((torch.linalg.vector_norm(out.double() - ref) / torch.linalg.vector_norm(ref)).item())
            row[prec] = {"ms_per_call": ms, "ops_per_s": w.K / (ms * 1e-3),
                         "tflops_logical": flops / (ms * 1e-3) / 1e12, "rel_fro_err_vs_fp64": err,
                         "kernels": kt}
        res[name] = row
        plan.close()
    return res


def run_blocked(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 200))
    res = blocked_report(steps, [args.precision] if args.precision else
                         ["bf16x3", "tf32", "fp32", "fp64"], flush)
    line = {"workload": "blocked U(1)xU(1), m=1000, d=4, K=200 (two sector laws)",
            "metric": "block-sparse rotation: ms per call, logical TFLOP/s over the realised problems",
            "steps": steps, "l2": "flushed between timed calls", "results": res, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def backward_report(steps, precs, flush):
    """The adjoint at the benchmark shape (d = 4, m = m' = 400, K = 150, FP32 operators,
    upstream G ~ N(0,1)): dO and dU per call for each precision, in forward-product
    equivalents (one forward product = 0.512 GFLOP logical per operator), with the
    error of the reduced paths against the FP32-input FP64 path."""
    import torch
    import paper_0909_5662_gb300 as P
    from workloads import dense_config, backward_upstream, SEED_BASE

    dev = flush.device
    w = dense_config(WORKLOAD)
    U = torch.from_numpy(w.U).to(dev)
    O32 = torch.from_numpy(w.O).to(dev, torch.float32)
    G32 = torch.from_numpy(backward_upstream(SEED_BASE + 4, w.K, w.mp)).to(dev, torch.float32)
    dO_ref, dU_ref = P.dmrg_rotate_ops_backward(U, O32.double(), G32.double(), w.d, "fp64")
    fwd_product = 2.0 * w.K * w.m * (w.d * w.mp) * w.m
    res = {}
    for prec in [p for p in precs if p != "fp64"]:
        dO, dU = P.dmrg_rotate_ops_backward(U, O32, G32, w.d, prec)
        ms = _timed(lambda: P.dmrg_rotate_ops_backward(U, O32, G32, w.d, prec), steps, 3, flush)
        P.dmrg_sync_status()
        num = torch.linalg.vector_norm((dO.double() - dO_ref).reshape(w.K, -1), dim=1)
        den = torch.linalg.vector_norm(dO_ref.reshape(w.K, -1), dim=1)
        res[prec] = {"ms_per_call": ms, "ops_per_s": w.K / (ms * 1e-3),
                     "forward_products_per_ms": 1.0 / ms,
                     "tflops_at_5_products": 5 * fwd_product / (ms * 1e-3) / 1e12,
                     "dO_max_rel_fro_err": float((num / den).max()),
                     "dU_rel_fro_err": float((torch.linalg.vector_norm(dU - dU_ref) /
                                              torch.linalg.vector_norm(dU_ref)).item())}
    if "fp64" in precs:
        t64 = _timed(lambda: P.dmrg_rotate_ops_backward(U, O32.double(), G32.double(), w.d, "fp64"),
                     1, 1, flush)
        res["fp64"] = {"ms_per_call": t64, "ops_per_s": w.K / (t64 * 1e-3)}
    return res


def run_backward(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 200))
    res = backward_report(steps, [args.precision] if args.precision else
                          ["bf16x3", "tf32", "fp32", "fp64"], flush)
    line = {"workload": "backward dense_m400_k150 (d=4, m=m'=400, K=150, upstream N(0,1))",
            "metric": "adjoint: ms per call (dO and dU), rotated operators/s",
            "steps": steps, "l2": "flushed between timed calls", "results": res, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def _kernel_report(timed_calls):
    """Per-kernel CUDA-event totals (ms per call and launches per call) over
    `timed_calls` calls, from the handle's kernel timing."""
    import paper_0909_5662_gb300 as P
    kt = P.dmrg_kernel_timing(reset=True)
    return {k["kernel"]: {"ms_per_call": k["total_ms"] / timed_calls,
                          "launches_per_call": k["launches"] / timed_calls,
                          "ms_per_launch": k["total_ms"] / k["launches"]} for k in kt}


def _with_kernel_timing(fn, calls, flush):
    """Runs fn `calls` times with per-kernel events on (L2 flushed before each call)."""
    import torch
    import paper_0909_5662_gb300 as P
    P.dmrg_kernel_timing(reset=True)
    P.dmrg_set_option("kernel_timing", 1)
    for _ in range(calls):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    P.dmrg_set_option("kernel_timing", 0)
    return _kernel_report(calls)


# FP64 arithmetic has no measured peak on this part: the denominator of FP64-bound
# kernels is the nominal GB300 rate (1.25 TFLOP/s, an FMA counted as 2 flops).
FP64_NOMINAL_GFLOPS = 1250.0


def run_truncation(args):
    """The truncation matrix (Sec. 2, steps 3-4): rho = Psi Psi^T of a superblock
    state with a ground-state-like Schmidt spectrum, its eigen-decomposition in FP64, the
    kept m' eigenvectors and the discarded weight.  Both solvers of the library (the
    default tridiagonal one and the cyclic Jacobi sweeps): time per call, per-kernel
    times, accuracy against the FP64 CPU oracle (the library eigh on the host cores),
    and the oracle's own time on the same state."""
    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    import oracle
    from workloads import schmidt_state, SEED_BASE

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 5))
    res = {}
    for n, mp in ((400, 100), (1600, 400)):
        name = "truncation_n%d_mp%d" % (n, mp)
        Psi_np = schmidt_state(SEED_BASE + 8, n, n)
        Psi = torch.from_numpy(Psi_np).to(dev)
        rho = Psi @ Psi.T
        if args.no_cpu_baseline:
            lam_ref, eps_ref, t_cpu = None, None, float("nan")
        else:
            t0 = time.perf_counter()
            U_ref, lam_ref, eps_ref = oracle.truncation(Psi_np, mp)
            t_cpu = time.perf_counter() - t0
        row = {"cpu_baseline": None if args.no_cpu_baseline else {
            "value": t_cpu * 1e3, "unit": "ms per call", "kind": "oracle", "cores": oracle.num_threads(),
            "sample": "the whole call: rho by rows, numpy.linalg.eigh, ranking"}}
        for method in ("tridiagonal", "jacobi"):
            h = P.Handle()
            P.dmrg_set_option("truncation_jacobi", 1 if method == "jacobi" else 0, handle=h)
            call = lambda: P.dmrg_truncation(Psi, mp, handle=h)
            U, lam, eps, sweeps = call()
            ms = _timed(call, steps, 1, flush)
            P.dmrg_kernel_timing(reset=True, handle=h)
            P.dmrg_set_option("kernel_timing", 1, handle=h)
            flush.zero_()
            call()
            torch.cuda.synchronize()
            P.dmrg_set_option("kernel_timing", 0, handle=h)
            kt = {k["kernel"]: {"ms_per_call": k["total_ms"], "launches_per_call": k["launches"]}
                  for k in P.dmrg_kernel_timing(reset=True, handle=h)}
            P.dmrg_sync_status(handle=h)
            resid = float(torch.linalg.vector_norm(rho @ U - U * lam[:mp][None, :], dim=0).max())
            ent = {"ms_per_call": ms, "sweeps": sweeps, "kernels": kt,
                   "max_residual_rhoU_minus_Ulambda": resid,
                   "orthonormality_err": float(torch.linalg.matrix_norm(
                       U.T @ U - torch.eye(mp, dtype=torch.float64, device=dev)).item()),
                   "eps": float(eps.item())}
            if lam_ref is not None:
                ent["max_abs_eig_err_vs_oracle"] = float(np.abs(lam.cpu().numpy() - lam_ref).max())
                ent["eps_abs_err_vs_oracle"] = abs(float(eps.item()) - eps_ref)
            if method == "jacobi" and "trunc_sweep" in kt:
                N = n + (n & 1)
                npair = N // 2
                # a rotation of a pair of entries is 6 flops: 4 per 2 x 2 block of A on the
                # upper triangle of pairs, 1 per (row, pair) of V; N - 1 rounds per sweep
                flops_sweep = (N - 1) * (24.0 * npair * (npair + 1) / 2 + 6.0 * n * npair)
                per = kt["trunc_sweep"]["ms_per_call"] / kt["trunc_sweep"]["launches_per_call"]
                gf = flops_sweep / (per * 1e-3) / 1e9
                ent["roofline"] = {"bound": "alu", "kernel": "trunc_sweep", "achieved": gf,
                                   "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s (FP64)",
                                   "frac": gf / FP64_NOMINAL_GFLOPS, "flops_per_launch": flops_sweep,
                                   "traffic": None, "peak_source": "nominal FP64 rate"}
            if method == "tridiagonal" and "trunc_tridiag" in kt:
                # Householder tridiagonalisation: 4 n^3 / 3 flops (multiply-adds counted as 2)
                gf = (4.0 * n ** 3 / 3.0) / (kt["trunc_tridiag"]["ms_per_call"] * 1e-3) / 1e9
                ent["roofline"] = {"bound": "alu", "kernel": "trunc_tridiag", "achieved": gf,
                                   "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s (FP64)",
                                   "frac": gf / FP64_NOMINAL_GFLOPS,
                                   "flops_per_launch": 4.0 * n ** 3 / 3.0, "traffic": None,
                                   "peak_source": "nominal FP64 rate"}
            row[method] = ent
            h.close()
        res[name] = row
    line = {"workload": "truncation of Schmidt-spectrum states (w_k ~ exp(-k/20)), "
                        "n = m d = 400 and 1600 rows, square Psi",
            "metric": "truncation matrix: ms per call (rho, eigen-decomposition, U, eps)",
            "steps": steps, "l2": "flushed between timed calls", "results": res, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_site(args):
    """Blocked site and cross operators O'_k = U^T ((A_k P^f) (x) S_c) U at d = 4,
    m = m' = 400, K = 150 (six Hubbard site-operator classes of 25): time per call
    for each precision, error against the FP64 GPU path, and the FP64 CPU oracle on
    a bounded sample (two operators per class)."""
    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    import oracle
    from workloads import site_workload

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 200))
    w = site_workload()
    U = torch.from_numpy(w.U).to(dev)
    A64 = torch.from_numpy(w.A).to(dev)
    A32 = A64.float()
    par = torch.from_numpy(w.parity).to(dev)
    call = lambda A, prec, out=None: P.dmrg_rotate_site_ops(U, A, w.d, w.S, w.counts, w.flags, par,
                                                            prec, out=out)
    ref = call(A32.double(), "fp64")
    flops = 2.0 * w.K * w.d * w.m * w.mp * (w.m + w.mp)
    res = {}
    precs = [args.precision] if args.precision else ["bf16x3", "tf32", "fp64"]
    for prec in precs:
        A = A32.double() if prec == "fp64" else A32
        out = call(A, prec)
        n = steps if prec != "fp64" else max(1, min(steps, 2))
        ms = _timed(lambda: call(A, prec, out), n, 3 if prec != "fp64" else 1, flush)
        kt = _with_kernel_timing(lambda: call(A, prec, out), min(n, 20), flush)
        P.dmrg_sync_status()
        num = torch.linalg.vector_norm((out.double() - ref).reshape(w.K, -1), dim=1)
        den = torch.linalg.vector_norm(ref.reshape(w.K, -1), dim=1)
        res[prec] = {"ms_per_call": ms, "ops_per_s": w.K / (ms * 1e-3),
                     "eff_tflops": flops / (ms * 1e-3) / 1e12,
                     "max_rel_fro_err_vs_fp64": float((num / den).max()), "kernels": kt}
    if args.no_cpu_baseline:
        print(json.dumps({"workload": "site_m400_k150", "results": res}), flush=True)
        return 0
    # the oracle on two operators of every class
    take = np.concatenate([np.arange(c * 25, c * 25 + 2) for c in range(len(w.counts))])
    t0 = time.perf_counter()
    o_ref = oracle.rotate_site(w.U, A32.double().cpu().numpy()[take], w.d, w.S,
                               np.full(len(w.counts), 2), w.flags, w.parity.astype(np.float64))
    t_cpu = time.perf_counter() - t0
    g = ref[torch.from_numpy(take).to(dev)].cpu().numpy()
    gpu_vs_oracle = float((np.linalg.norm((g - o_ref).reshape(len(take), -1), axis=1) /
                           np.linalg.norm(o_ref.reshape(len(take), -1), axis=1)).max())
    line = {"workload": "site_m400_k150 (d=4, m=m'=400, K=150: c_up, c_dn, c+_up, c+_dn with the "
                        "block parity, n_up, n_dn; 25 block operators each)",
            "metric": "blocked site/cross operators: ms per call, rotated operators/s",
            "steps": steps, "l2": "flushed between timed calls", "results": res,
            "fp64_gpu_vs_oracle_max_rel_fro": gpu_vs_oracle,
            "cpu_baseline": {"value": len(take) / t_cpu, "unit": "rotated operators/s",
                             "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": "%d operators (2 per class), FP64 loops" % len(take)},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_fused(args):
    """The fused rotation (both products of Sec. 3.2 in one kernel, the intermediate
    (O_k (x) I_d) U kept in tensor memory and shared memory) against the two-product
    path: BF16x3, d = 4, m = 400, K = 150, m' = 64, 128, 256 (the fused kernel holds
    at most 256 output columns).  Time per call, kernel times, the fused kernel's
    issued tensor-core rate, and the error of both against the FP64 oracle on sampled
    operators."""
    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    import oracle
    from workloads import dense_workload, SEED_BASE

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 200))
    peaks, peak_src = measured_peaks()
    m, d, K = 400, 4, 150
    sample = [0, 74, 149]
    res = {}
    t_cpu = 0.0
    for mp in (64, 128, 256):
        w = dense_workload("fused", SEED_BASE + 20 + mp, d, m, mp, K)
        U = torch.from_numpy(w.U).to(dev)
        O32 = torch.from_numpy(w.O).to(dev, torch.float32)
        t0 = time.perf_counter()
        ref = oracle.rotate_dense(w.U, w.O.astype(np.float32).astype(np.float64)[sample], d)
        t_cpu += time.perf_counter() - t0
        entry = {}
        for name, fused in (("two_products", 0), ("fused", 1)):
            P.dmrg_set_option("fused_rotation", fused)
            out = P.dmrg_rotate_ops(U, O32, d, "bf16x3")
            ms = _timed(lambda: P.dmrg_rotate_ops(U, O32, d, "bf16x3", out=out), steps, 3, flush)
            kt = _with_kernel_timing(lambda: P.dmrg_rotate_ops(U, O32, d, "bf16x3", out=out),
                                     min(steps, 20), flush)
            P.dmrg_sync_status()
            got = out[sample].double().cpu().numpy()
            err = np.linalg.norm((got - ref).reshape(len(sample), -1), axis=1) / \
                np.linalg.norm(ref.reshape(len(sample), -1), axis=1)
            entry[name] = {"ms_per_call": ms, "ops_per_s": K / (ms * 1e-3), "kernels": kt,
                           "max_rel_fro_err_vs_oracle": float(err.max())}
        P.dmrg_set_option("fused_rotation", 0)
        fk = entry["fused"]["kernels"].get("tc_fused_rotation")
        if fk:
            issued = 3.0 * 2.0 * K * d * m * mp * (m + mp)
            ach = issued / (fk["ms_per_launch"] * 1e-3) / 1e12
            entry["fused"]["roofline"] = {
                "bound": "tensor", "kernel": "tc_fused_rotation", "achieved": ach,
                "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": ach / peaks["bf16_tflops"],
                "traffic": None, "flops_per_launch": issued,
                "peak_source": "%s bf16_tflops (burst)" % peak_src}
        res["mp%d" % mp] = entry
    line = {"workload": "fused_m400_k150 (d=4, m=400, K=150, m'=64/128/256, BF16x3, FP32 operators)",
            "metric": "dense rotation: ms per call, fused kernel vs the two products",
            "steps": steps, "l2": "flushed between timed calls", "results": res,
            "cpu_baseline": {"value": 3 * len(sample) / t_cpu, "unit": "rotated operators/s",
                             "kind": "oracle", "cores": oracle.num_threads(),
                             "sample": "%d operators at each m', FP64" % len(sample)},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


def run_measure(args):
    """The measurement stage on the superblock state of the m = 400, d = 4 step
    (Psi 1600 x 1600): <Z_k> for 150 system operators (rho = Psi Psi^T, then
    Tr(rho Z_k)), the 50 x 50 system-environment correlations, and N(q) at L = 128.
    Time per call, per-kernel times, and the FP64 CPU oracle on a bounded sample."""
    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    import oracle
    from workloads import measure_workload

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    steps = max(1, min(args.steps, 20))
    w = measure_workload()
    Psi = torch.from_numpy(w.Psi).to(dev)
    Z = torch.from_numpy(w.Z).to(dev)
    W = torch.from_numpy(w.W).to(dev)
    G = torch.from_numpy(w.G).to(dev)
    v = torch.from_numpy(w.v).to(dev)
    n = w.Psi.shape[0]
    Ks, Ke = Z.shape[0], W.shape[0]
    Zc = Z[:Ke].contiguous()          # correlations: the first Ke system operators
    res = {}
    calls = {
        "expectation": lambda: P.dmrg_expectation(Z, Psi, 0),
        "cross_correlations": lambda: P.dmrg_cross_correlations(Zc, W, Psi),
        "structure_factor": lambda: P.dmrg_structure_factor(G, v, 0.5),
    }
    for name, fn in calls.items():
        got = fn()
        ms = _timed(fn, steps, 2, flush)
        kt = _with_kernel_timing(fn, min(steps, 5), flush)
        P.dmrg_sync_status()
        res[name] = {"ms_per_call": ms, "kernels": kt}
    peaks, peak_src = measured_peaks()
    tr = res["expectation"]["kernels"].get("measure_trace")
    if tr:
        gbs = (Ks * n * n * 4 + n * n * 8) / (tr["ms_per_launch"] * 1e-3) / 1e9
        res["expectation"]["roofline_trace"] = {
            "bound": "hbm", "kernel": "measure_trace", "achieved": gbs, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None,
            "bytes_per_launch": Ks * n * n * 4 + n * n * 8, "peak_source": "%s hbm_gbs" % peak_src}
    rh = res["expectation"]["kernels"].get("measure_rho")
    if rh:
        # rho is symmetric: n(n+1)/2 distinct entries, 2n flops each
        flops = float(n) * (n + 1) * n
        gf = flops / (rh["ms_per_launch"] * 1e-3) / 1e9
        res["expectation"]["roofline_rho"] = {
            "bound": "alu", "kernel": "measure_rho", "achieved": gf, "peak": FP64_NOMINAL_GFLOPS,
            "unit": "GFLOP/s (FP64)", "frac": gf / FP64_NOMINAL_GFLOPS, "traffic": None,
            "flops_per_launch": flops,
            "peak_source": "nominal FP64 rate (no measured FP64 peak)"}
    if args.no_cpu_baseline:
        print(json.dumps({"workload": "measure_m400", "results": res}), flush=True)
        return 0
    # accuracy and the oracle on a bounded sample
    take = 4
    t0 = time.perf_counter()
    e_ref = oracle.expectation(w.Z[:take].astype(np.float64), w.Psi, 0)
    t_cpu = time.perf_counter() - t0
    e_gpu = P.dmrg_expectation(Z[:take].contiguous(), Psi, 0).cpu().numpy()
    c_ref = oracle.cross_correlations(w.Z[:2].astype(np.float64), w.W[:2].astype(np.float64), w.Psi)
    c_gpu = P.dmrg_cross_correlations(Z[:2].contiguous(), W[:2].contiguous(), Psi).cpu().numpy()
    f_ref = oracle.structure_factor(w.G, w.v, 0.5)
    f_gpu = [x.cpu().numpy() for x in P.dmrg_structure_factor(G, v, 0.5)]
    line = {"workload": "measure_m400 (Psi 1600 x 1600 with w_k ~ exp(-k/20); 150 system "
                        "operators for <Z>, 50 x 50 for the correlations, FP32; L = 128 "
                        "structure factor)",
            "metric": "measurement stage: ms per call",
            "steps": steps, "l2": "flushed between timed calls", "results": res,
            "max_abs_err_vs_oracle": {
                "expectation": float(np.abs(e_gpu - e_ref).max()),
                "cross_correlations": float(np.abs(c_gpu - c_ref).max()),
                "structure_factor": float(max(np.abs(f_gpu[0] - f_ref[0]).max(),
                                              np.abs(f_gpu[1] - f_ref[1]).max()))},
            "cpu_baseline": {"value": take / t_cpu, "unit": "expectation values/s", "kind": "oracle",
                             "cores": oracle.num_threads(),
                             "sample": "%d of the 150 system operators: rho and Tr(rho Z), FP64 loops" % take},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------- chained sweep
def chained_report(sweep_steps, with_oracle):
    """50 consecutive block-growth steps at d = 4, m = m' = 1200, K = 300: the rotated
    operators of step s are the inputs of step s + 1, with a fresh seeded orthonormal U
    per step.  BF16x3 and TF32 carry all 300 operators; the FP64 GPU path carries a
    tracked subset (operators are independent given U) as the drift reference, and its
    first step is checked against the FP64 CPU oracle.  At the end the FP64 two-point
    functions <psi|O'_i O'_j|psi> of the tracked operators are compared."""
    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    from workloads import chained_inputs, SEED_BASE

    dev = torch.device("cuda", torch.cuda.current_device())
    d, m, K = 4, 1200, 300
    steps = sweep_steps
    track = list(range(0, K, K // 16))[:16]
    g = torch.Generator(device=dev)
    g.manual_seed(SEED_BASE + 5)
    O0 = torch.randn(K, m, m, generator=g, dtype=torch.float64, device=dev)
    psi = torch.randn(m, generator=g, dtype=torch.float64, device=dev)
    psi /= torch.linalg.vector_norm(psi)
    cur = {"bf16x3": O0.float(), "tf32": O0.float()}
    ref = O0[track].clone()
    outs = {p: torch.empty_like(cur[p]) for p in cur}
    ref_out = torch.empty_like(ref)
    drift = {p: [] for p in cur}
    ms = {p: 0.0 for p in cur}
    oracle_step1 = None
    for step in range(steps):
        U = chained_inputs(step, m * d, m, dev)
        for p in cur:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            P.dmrg_rotate_ops(U, cur[p], d, p, out=outs[p])
            b.record()
            b.synchronize()
            ms[p] += a.elapsed_time(b)
            cur[p], outs[p] = outs[p], cur[p]
        P.dmrg_rotate_ops(U, ref, d, "fp64", out=ref_out)
        ref, ref_out = ref_out, ref
        P.dmrg_sync_status()
        if step == 0 and with_oracle:
            import oracle
            sub = [0, 1]
            r0 = oracle.rotate_dense(U.cpu().numpy(), O0[[track[i] for i in sub]].cpu().numpy(), d)
            num = np.linalg.norm((ref[sub].cpu().numpy() - r0).reshape(len(sub), -1), axis=1)
            oracle_step1 = float((num / np.linalg.norm(r0.reshape(len(sub), -1), axis=1)).max())
        for p in cur:
            x = cur[p][track].double()
            num = torch.linalg.vector_norm((x - ref).reshape(len(track), -1), dim=1)
            den = torch.linalg.vector_norm(ref.reshape(len(track), -1), dim=1)
            drift[p].append(float((num / den).max()))
    C_ref = P.dmrg_correlations(ref, psi)
    corr = {}
    for p in cur:
        C = P.dmrg_correlations(cur[p][track].contiguous(), psi)
        corr[p] = float((torch.linalg.vector_norm(C - C_ref) / torch.linalg.vector_norm(C_ref)).item())
    flops_step = 2.0 * K * d * m * m * (m + m)
    return {"workload": "chained_m1200_k300 (d=4, m=m'=1200, K=300, %d steps)" % steps,
            "metric": "chained sweep: rotated operators/s per precision, accumulated drift",
            "unit": UNIT, "steps": steps,
            "precisions": {p: {"ms_per_step": ms[p] / steps,
                               "ops_per_s": K / (ms[p] / steps * 1e-3),
                               "eff_tflops": flops_step / (ms[p] / steps * 1e-3) / 1e12,
                               "max_rel_fro_drift_first": drift[p][0],
                               "max_rel_fro_drift_last": drift[p][-1],
                               "drift_per_step": drift[p],
                               "correlation_rel_err": corr[p]} for p in cur},
            "fp64_reference": {"tracked_operators": track, "oracle_step1_rel_err": oracle_step1},
            "data": "synthetic"}


def run_chained(args):
    import torch
    torch.cuda.set_device(0)
    print(json.dumps(chained_report(args.sweep_steps, not args.no_cpu_baseline)), flush=True)
    return 0


def dtype_peaks(dev):
    """Measured dense matmul peaks of the other two precisions the rotation runs in:
    TF32 (FP32 torch.matmul with TF32 tensor cores allowed, 8192^3) and FP64
    (torch.matmul, 4096^3), best of several calls timed with CUDA events.  No clock or
    power setting is touched."""
    import torch
    out = {}
    for name, dt, n, reps in (("tf32_tflops", torch.float32, 8192, 10),
                              ("fp64_tflops", torch.float64, 4096, 4)):
        old = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = (dt == torch.float32)
        try:
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            c = a @ b
            torch.cuda.synchronize()
            best = 1e30
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            out[name.replace("_tflops", "_how")] = "torch.matmul %d^3, best of %d (CUDA events)" % (n, reps)
            del a, b, c
        finally:
            torch.backends.cuda.matmul.allow_tf32 = old
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="dense line only: skip the blocked, backward and chained reports and "
                         "the TF32/FP64 matmul peaks")
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "chained", "blocked", "backward", "site", "measure", "truncation",
                             "fused"],
                    help="dense: the benchmark line; chained: the 50-step sweep report; "
                         "blocked / backward / site / measure / truncation / fused: reports of "
                         "the block-sparse, adjoint, site-operator, measurement, truncation and "
                         "fused-rotation paths")
    ap.add_argument("--precision", default=None, choices=["bf16x3", "tf32", "fp32", "fp64"],
                    help="blocked / backward / site reports: time this precision only")
    ap.add_argument("--sweep-steps", type=int, default=50)
    ap.add_argument("--profile", action="store_true",
                    help="only the BF16x3 step: warm-up then --steps steps (for ncu captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "chained":
        return run_chained(args)
    if args.workload == "blocked":
        return run_blocked(args)
    if args.workload == "backward":
        return run_backward(args)
    if args.workload == "site":
        return run_site(args)
    if args.workload == "measure":
        return run_measure(args)
    if args.workload == "truncation":
        return run_truncation(args)
    if args.workload == "fused":
        return run_fused(args)

    import numpy as np
    import torch
    import paper_0909_5662_gb300 as P
    from paper_0909_5662_gb300 import umd_partition
    from workloads import dense_workload, SEED_BASE

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    # Weak scaling: the job holds K_PER_GPU * ws operators, UMD-partitioned.
    K_total = K_PER_GPU * ws
    lo, hi = umd_partition(K_total, ws, rank)
    # every rank's slice has the same shape and statistics; ranks > 0 shift the seed
    w = dense_workload(WORKLOAD, SEED_BASE + 2 + 1000 * rank, D, M, MP, hi - lo, hubbard_mix=True)
    K = w.K
    U = torch.from_numpy(w.U).to(dev)
    O32 = torch.from_numpy(w.O).to(dev, torch.float32)
    O64 = torch.from_numpy(w.O).to(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    h = P.default_handle()
    flops_logical = 2.0 * K * D * M * MP * (M + MP)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def time_steps(prec, O, steps, warmup, timing=False, sampler=None):
        out = P.dmrg_rotate_ops(U, O, D, prec)
        for _ in range(warmup):
            P.dmrg_rotate_ops(U, O, D, prec, out=out)
        barrier()
        if sampler is not None:
            sampler.mark("t_begin")
        if timing:
            P.dmrg_kernel_timing(reset=True)
            P.dmrg_set_option("kernel_timing", 1)
        evs = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            P.dmrg_rotate_ops(U, O, D, prec, out=out)
            b.record()
            evs.append((a, b))
        barrier()
        if sampler is not None:
            sampler.mark("t_end")
        if timing:
            P.dmrg_set_option("kernel_timing", 0)
        per = [a.elapsed_time(b) for a, b in evs]
        ms = sum(per)
        kt = P.dmrg_kernel_timing(reset=True) if timing else []
        P.dmrg_sync_status()
        time_steps.last_median = sorted(per)[len(per) // 2] if per else 0.0
        return ms, kt, out

    if args.profile:
        out = P.dmrg_rotate_ops(U, O32, D, "bf16x3")
        for _ in range(args.warmup + args.steps):
            P.dmrg_rotate_ops(U, O32, D, "bf16x3", out=out)
        torch.cuda.synchronize()
        P.dmrg_sync_status()
        print(json.dumps({"profile": WORKLOAD, "steps": args.steps, "warmup": args.warmup}))
        return 0

    def max_over_ranks(x):
        if pg is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        return float(t.item())

    # ---- headline: BF16x3, clocks sampled during the timed region
    sampler = ClockSampler(local if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    P.dmrg_rotate_ops(U, O32, D, "bf16x3")
    torch.cuda.synchronize()
    sampler.start()
    ms_total, _, out_bf = time_steps("bf16x3", O32, args.steps, args.warmup, timing=False,
                                     sampler=sampler)
    clocks = sampler.stop()
    ms_step = max_over_ranks(ms_total / args.steps)
    value = K_total / (ms_step * 1e-3)
    # Per-kernel durations for the roofline come from a second loop of the same steps
    # (same L2 flushes) with CUDA events around every kernel launch; those events
    # serialise the launches, so this loop is not the one the headline is timed on.
    ms_instr, kt, _ = time_steps("bf16x3", O32, args.steps, args.warmup, timing=True)
    launches_per_step = sum(k["launches"] for k in kt) / max(args.steps, 1)

    # ---- dominant kernel roofline (issued BF16 MMA flops: 3 per logical multiply-add pair)
    peaks, peak_src = measured_peaks()
    per_kernel = {k["kernel"]: k["total_ms"] / k["launches"] for k in kt}
    dom = max(per_kernel, key=per_kernel.get)
    issued = {"tc_gemm_first_product": 3 * 2.0 * K * M * (D * MP) * M,
              "tc_gemm_second_product": 3 * 2.0 * K * MP * MP * (M * D)}
    if dom in issued:
        achieved = issued[dom] / (per_kernel[dom] * 1e-3) / 1e12
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for(dom), "kernel": dom,
                "peak_source": "%s bf16_tflops (burst)" % peak_src,
                "flops_per_launch": issued[dom], "ms_per_launch": per_kernel[dom]}
    else:
        byt = {"pack_operands": K * M * M * (4 + 4),
               "pack_u": D * M * MP * 8 + 2 * (2 * D * M * MP * 2)}
        achieved = byt.get(dom, 0) / (per_kernel[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic_for(dom), "kernel": dom}

    # ---- the same inputs in TF32 and through the plain FP64 GPU path
    # The side precisions report the median step: one host stall inside one call of the
    # 20 (seen once, about 40 ms) would otherwise decide their mean.
    ms_tf, _, out_tf = time_steps("tf32", O32, args.steps, args.warmup, timing=False)
    ms_tf = time_steps.last_median * args.steps
    fp64_steps = 2
    ms_64, _, out_64 = time_steps("fp64", O64, fp64_steps, 1)
    ms_tf = max_over_ranks(ms_tf / args.steps)
    ms_64 = max_over_ranks(ms_64 / fp64_steps)

    # ---- accuracy of the reduced paths against the FP64 GPU path (oracle-checked in tests)
    def rel(a, b):
        num = torch.linalg.vector_norm((a.double() - b).reshape(K, -1), dim=1)
        den = torch.linalg.vector_norm(b.reshape(K, -1), dim=1)
        return float((num / den).max())
    err_bf = rel(out_bf, out_64)
    err_tf = rel(out_tf, out_64)

    # ---- end to end through the public API with host buffers (pinned): one
    #      dmrg_rotate_ops_host call per step copies the operators in, rotates them
    #      and copies the result out, overlapping the three in chunks.
    Oh = torch.from_numpy(w.O.astype(np.float32)).pin_memory()
    Uh = torch.from_numpy(w.U).pin_memory()
    outh = torch.empty((K, MP, MP), dtype=torch.float32).pin_memory()
    for _ in range(args.warmup):
        P.dmrg_rotate_ops_host(Uh, Oh, D, "bf16x3", out=outh, synchronize=False)
    barrier()
    e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        P.dmrg_rotate_ops_host(Uh, Oh, D, "bf16x3", out=outh, synchronize=False)
        b.record()
        b.synchronize()
        e_ms += a.elapsed_time(b)
    e_ms = max_over_ranks(e_ms / args.steps)
    h2d = Oh.numel() * 4 + Uh.numel() * 8
    d2h = outh.numel() * 4
    e2e_err = rel(outh.to(dev), out_64)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(w)

    # ---- the other workloads of the method on one GPU (block-sparse, adjoint, chained
    #      sweep) and the TF32 / FP64 matmul peaks, after every timed dense step
    extras = {}
    if rank == 0 and ws == 1 and not args.no_extras:
        del out_bf, out_tf, out_64
        torch.cuda.empty_cache()
        n_extra = max(3, min(args.steps, 50))
        pk = dtype_peaks(dev)
        eff_tf = flops_logical / (ms_tf * 1e-3) / 1e12
        eff_64 = flops_logical / (ms_64 * 1e-3) / 1e12
        extras["dtype_peaks"] = dict(pk, bf16_tflops=peaks["bf16_tflops"],
                                     bf16_source="%s bf16_tflops (burst)" % peak_src)
        extras["precision_fractions"] = {
            "bf16x3_issued_of_bf16_peak": 3 * flops_logical / (ms_step * 1e-3) / 1e12 / peaks["bf16_tflops"],
            "tf32_of_tf32_peak": eff_tf / pk["tf32_tflops"],
            "fp64_of_fp64_peak": eff_64 / pk["fp64_tflops"],
            "note": "whole-step rates (all kernels of the step) over the measured matmul peak "
                    "of the precision the products issue: BF16x3 issues 3 BF16 MMAs per "
                    "logical multiply-add, TF32 one, FP64 (SIMT FMA) one"}
        extras["blocked"] = blocked_report(n_extra, ["bf16x3", "tf32", "fp32", "fp64"], flush)
        extras["backward"] = backward_report(n_extra, ["bf16x3", "tf32", "fp32", "fp64"], flush)
        extras["chained"] = chained_report(args.sweep_steps, not args.no_cpu_baseline)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
            "config": {
                "workload": "%s (d=4, m=400 -> m*d=1600 -> m'=400, K=150 per GPU)" % WORKLOAD,
                "precision": "BF16x3 (bf16 hi/lo operands, fp32 accumulate), output fp32",
                "operators_total": K_total, "partition": "UMD contiguous slices, no collective",
                "l2": "flushed between timed steps (512 MiB write, not timed)",
                "kernel_timing": "per-kernel CUDA events in a second loop of the same steps "
                                 "(%.4f ms/step with them)" % (ms_instr / args.steps),
                "inputs": "resident in HBM (operators fp32, U fp64)"},
            "eff_tflops": flops_logical / (ms_step * 1e-3) / 1e12 * 1.0,
            "issued_bf16_tflops": 3 * flops_logical / (ms_step * 1e-3) / 1e12,
            "precisions": {
                "bf16x3": {"ms_per_step": ms_step, "ops_per_s": K_total / (ms_step * 1e-3),
                           "eff_tflops": flops_logical / (ms_step * 1e-3) / 1e12,
                           "max_rel_fro_err_vs_fp64": err_bf},
                "tf32": {"ms_per_step": ms_tf, "step_statistic": "median of the timed steps",
                         "ops_per_s": K_total / (ms_tf * 1e-3),
                         "eff_tflops": flops_logical / (ms_tf * 1e-3) / 1e12,
                         "max_rel_fro_err_vs_fp64": err_tf},
                "fp64": {"ms_per_step": ms_64, "ops_per_s": K_total / (ms_64 * 1e-3),
                         "eff_tflops": flops_logical / (ms_64 * 1e-3) / 1e12}},
            "kernels_ms_per_launch": per_kernel,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": K_total / (e_ms * 1e-3), "unit": UNIT, "ms_per_step": e_ms,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "dmrg_rotate_ops_host (pinned host buffers, chunked copy/compute overlap)",
                    "max_rel_fro_err_vs_fp64": e2e_err},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
