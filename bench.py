#!/usr/bin/env python
"""Benchmark of the LADMM solver on one GB300 (or N replicas under torchrun).

Metric: voxel x compartment x iterations per second of the LADMM iteration
(Algorithm 2), plus time to tolerance (p50/p99), per precision form, on the 2D
diffusion-relaxation slice workload: 128 x 128 voxels (N = 16384), P = 120 encodings
(15 b-values x 8 echo times), Q = 2500 compartments (50 x 50 log-spaced D x T2),
lambda = 1e-2, synthetic seeded data (SNR 100).

A step is one ssm_solve: the data projections (Algorithm 2, step 4), ITERS_PER_STEP
iterations of steps 6-11 with the residual test every 10 iterations, and the copy of
z into F. The plan (steps 1-3: Gram, eigendecomposition, rank, weights) is built once
per dictionary before the timed region; its time is reported as plan_ms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own independent problem (a different seed) with
no collective on the data path: weak scaling, value = all ranks' work / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "dr2d_slice"


def describe(w):
    if w.name == "dr2d_slice":
        return "2D diffusion-relaxation slice 128x128"
    return f"{len(w.dims)}D grid {'x'.join(str(d) for d in w.dims)}"
ITERS_PER_STEP = 100
CHECK_EVERY = 10
TTT_TOL = 3e-4
METRIC = "voxel*compartment*iters/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto",
                    help="headline form: lowrank_tf32x3 | lowrank_fp32 | dense_bf16x3 | "
                         "dense_fp32 | admm_fp32 | auto (the form with the lowest time to "
                         "the objective gap 1e-4)")
    ap.add_argument("--ttt-repeats", type=int, default=20,
                    help="fresh solves to the residual rule per low-rank form (p50/p99)")
    ap.add_argument("--ref-iters", type=int, default=REF_ITERS,
                    help="iterations of the reference run for the objective gap and DFCS")
    ap.add_argument("--trace-budget", type=float, default=TRACE_BUDGET_S,
                    help="GPU seconds per form for the objective-gap / DFCS trace")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline form only")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving run")
    ap.add_argument("--no-batching", action="store_true", help="skip the batching run")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the per-iteration lines of the 3D and fingerprinting workloads")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="workload of the timed steps (default: the 128x128 slice the metric "
                         "is quoted on; the others serve profiling)")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-iters", type=int, default=100,
                    help="iterations per served request (a fixed budget)")
    ap.add_argument("--serve-load", type=float, default=0.7,
                    help="Poisson arrival rate as a fraction of the measured capacity")
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    PERIOD_MS = 100

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None
        self.skip = 0

    def start(self):
        """Start sampling and return once the sampler has taken its first sample (its
        start-up would otherwise fall inside a short timed region); that sample and any
        other taken before this returns are dropped."""
        self.skip = 0
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            lines = self._lines()
            if lines:
                self.skip = len(lines)
                return
            time.sleep(0.01)

    def _lines(self):
        self.tmp.flush()
        with open(self.tmp.name) as f:
            return [ln for ln in f.read().splitlines() if ln.strip()]

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lines = self._lines()
        os.unlink(self.tmp.name)
        # the samples taken once the timed region had begun; a region shorter than one
        # period reports the sample taken just before it
        rows = [ln.split(",") for ln in lines[min(self.skip, max(len(lines) - 1, 0)):]]
        sms, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sms.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sms:
            out = {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(mx),
                   "reasons": sorted(reasons), "samples": len(sms),
                   "power_w_max": max(power) if power else None}
        return out


# --------------------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------------------
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def traffic_record(kernel_file, kernel_name, workload=None):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is
    unchanged since the capture (profiles/traffic.json records its hash) and the capture
    was of the workload being run."""
    workload = workload or WORKLOAD
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[
            f"{kernel_name} @ {workload}"]
    except (OSError, ValueError, KeyError):
        return None
    src = os.path.join(ROOT, "paper_2401_12890_gb300", "csrc", kernel_file)
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha") != h or rec.get("bench_workload", "dr2d_slice") != workload:
        return None
    return rec.get("dram_bytes_per_launch_full")


def weak_value(world, N, Q, seconds_per_step):
    """Whole-job throughput under weak scaling: every rank solves its own problem of N
    voxels and Q compartments, ITERS_PER_STEP iterations per step, and a step takes as
    long as the slowest rank's (the max over ranks)."""
    return world * N * Q * ITERS_PER_STEP / seconds_per_step


def rank_seed(base_seed, rank):
    """Each rank's own synthetic problem: the workload's seed offset by the rank."""
    return base_seed + 7919 * rank


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, backend):
        self.world, self.rank, self.local = dist_env()
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v):
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


FORMS = [("lowrank", "tf32x3"), ("lowrank", "fp32"), ("dense", "bf16x3"), ("dense", "fp32"),
         ("admm", "fp32")]
# time to tolerance by the objective gap (J - J_ref) / J_ref and by DFCS (Eq. 33)
GAP_TOLS = (1e-3, 1e-4)
DFCS_TOL = 1e-2
REF_ITERS = 60000          # the reference run (full-rank BF16x3 form)
TRACE_BLOCK = 500          # iterations between objective evaluations of a trace
TRACE_BUDGET_S = 12.0      # GPU seconds a form's trace may take


def form_key(form, prec):
    return f"{form}_{prec}"


def trace_to_tolerance(plan, Md, F, J_full, f_ref, J_ref, budget_s, max_iters, stream):
    """One solve continued block by block (ssm_solve_resume): after each block of
    TRACE_BLOCK iterations, the objective with the full K and DFCS = ||z - f_ref|| /
    ||f_ref|| (Eq. 33). Returns the device time at which each tolerance was first met
    (block granularity; None if not within the budget), and the last values."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.set_max_iter(TRACE_BLOCK)
    t_gpu, k = 0.0, 0
    hit_gap = {tol: None for tol in GAP_TOLS}
    hit_dfcs = None
    nref = float(torch.linalg.vector_norm(f_ref)) if f_ref is not None else None
    gap = dfcs = None
    curve = []
    first = True
    while k < max_iters and t_gpu < budget_s:
        e0.record(stream)
        if first:
            plan.solve_async(Md, F)
            first = False
        else:
            plan.resume(Md, F)
        e1.record(stream)
        torch.cuda.synchronize()
        t_gpu += e0.elapsed_time(e1) / 1e3
        k += TRACE_BLOCK
        J = J_full(F)
        if J_ref is not None:
            gap = (J - J_ref) / J_ref
            for tol in GAP_TOLS:
                if hit_gap[tol] is None and gap <= tol:
                    hit_gap[tol] = {"ms": 1e3 * t_gpu, "iterations": k}
        if f_ref is not None:
            dfcs = float(torch.linalg.vector_norm(F - f_ref)) / nref
            if hit_dfcs is None and dfcs <= DFCS_TOL:
                hit_dfcs = {"ms": 1e3 * t_gpu, "iterations": k}
        if len(curve) < 64 and (k // TRACE_BLOCK) in (1, 2, 4, 8, 16, 32, 64, 128):
            curve.append({"iterations": k, "ms": 1e3 * t_gpu, "objective_gap": gap,
                          "dfcs": dfcs})
        if all(v is not None for v in hit_gap.values()) and (f_ref is None or hit_dfcs):
            break
    return {"gap": {f"{tol:g}": hit_gap[tol] for tol in GAP_TOLS}, "dfcs": hit_dfcs,
            "curve": curve,
            "last": {"iterations": k, "gpu_ms": 1e3 * t_gpu, "objective_gap": gap,
                     "dfcs": dfcs, "objective_full_k": J}}


def dominant_kernel(form, prec, Q, N, r, fused=0):
    """(kernel name, source file, bound, algorithmic amount per launch, unit, traffic key).

    The tensor-core form runs one of three forms, whichever the plan's autotuner measured
    fastest: the GEMM + update pair, or the fused kernel (the GEMM with the update in its
    epilogue: the whole iteration) with a staged (1) or register (2) epilogue. Its
    dominant kernel is the GEMM either way, and its bound the tensor-core flops."""
    if form == "lowrank":
        # read z and write z' per state element (d cancels from the iteration, see
        # ssm_lowrank.cu); read S, u and write u' per voxel
        if prec == "tf32x3":
            return ("lrtc_kernel", "ssm_lowrank_tc.cu", "hbm", 8.0 * Q * N + 12.0 * r * N,
                    "GB/s", "lrtc_kernel")
        return ("lowrank_iter_kernel", "ssm_lowrank.cu", "hbm",
                8.0 * Q * N + 12.0 * r * N, "GB/s", "lowrank_iter_kernel")
    if prec == "fp32":
        # (for Algorithm 1 the profiled time is the whole iteration, of which the x-step
        # product is this amount of work)
        return ("sgemm_kernel", "ssm_dense.cu", "alu", 2.0 * Q * Q * N, "TFLOP/s", "sgemm_kernel")
    key = {0: "tc_gemm_kernel", 1: "tc_gemm_kernel (fused, staged epilogue)",
           2: "tc_gemm_kernel (fused, register epilogue)"}[fused]
    return ("tc_gemm_kernel", "ssm_tc.cu", "tensor", 3 * 2.0 * Q * Q * N, "TFLOP/s", key)


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def bench_ours(args):
    import torch

    import __graft_entry__
    from paper_2401_12890_gb300 import ssm, synth

    dist = Dist("nccl")
    torch.cuda.set_device(dist.local)
    if dist.rank == 0:
        __graft_entry__.build()
    dist.barrier()
    ssm.load_library()
    w = synth.WORKLOADS[WORKLOAD]
    K, M, _ = synth.make_problem(WORKLOAD, seed=rank_seed(w.seed, dist.rank))
    N, Q, P = w.N, w.Q, w.P
    Md = torch.from_numpy(M).cuda()
    F = torch.empty((Q, N), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def make_plan(form, prec, **kw):
        base = dict(form=form, precision=prec, max_iter=ITERS_PER_STEP, check_every=CHECK_EVERY)
        base.update(kw)
        return ssm.Plan(K, w.dims, w.lam, w.beta, **base)

    # which forms this build offers
    available = []
    for form, prec in FORMS:
        try:
            pl = make_plan(form, prec, max_iter=1)
            pl.close()
            available.append((form, prec))
        except ssm.SsmError as e:
            if e.status != ssm.SSM_EUNSUPPORTED:
                raise

    results = {}
    # The reference for time to tolerance (objective gap and DFCS, Eq. 33): the paper's
    # f* is the converged iterate of the unapproximated problem; here it is the full-rank
    # BF16x3 form after REF_ITERS iterations, computed on this GPU in this run (the FP64
    # oracle cannot converge this workload on the host: its objective still falls by
    # ~5e-5 per doubling of the iteration count after 32000 iterations).
    ref_form = ("dense", "bf16x3") if ("dense", "bf16x3") in available else ("dense", "fp32")
    reference = None
    f_ref = J_ref = None
    if not args.quick:
        rplan = make_plan(*ref_form, max_iter=args.ref_iters, check_every=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f_ref, _ = rplan.solve(Md)
        torch.cuda.synchronize()
        J_ref = rplan.objective(Md, f_ref, use_full_k=True)
        reference = {"form": form_key(*ref_form), "iterations": args.ref_iters,
                     "objective_full_k": J_ref, "seconds": time.perf_counter() - t0,
                     "note": "J_ref and f_ref of the objective-gap and DFCS tolerances: "
                             "computed on the GPU in this run; the remaining decrease after "
                             "this many iterations is of order 1e-5 of J"}
        rplan.close()

    def J_full_of(plan):
        return lambda Fz: plan.objective(Md, Fz, use_full_k=True)

    ttt = {}
    explicit = None if args.form == "auto" else tuple(args.form.split("_"))
    # --quick with a named form: that form alone (profiling runs)
    ttt_forms = [explicit] if (args.quick and explicit in available) else available
    for form, prec in ttt_forms:
        key = form_key(form, prec)
        rec = {}
        # time to tolerance by the paper's residual rule: fresh solves to ||z-f|| and
        # ||dz|| <= TTT_TOL ||z||, repeated (p50/p99 over the samples)
        tplan = make_plan(form, prec, max_iter=20000, tol_primal=TTT_TOL, tol_change=TTT_TOL)
        slow = prec == "fp32" and form != "lowrank"   # seconds per solve: one cold sample
        reps = 1 if slow else (args.ttt_repeats if form == "lowrank" else 5)
        if not slow:
            tplan.solve(Md, F)
        times, iters = [], []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, tinfo = tplan.solve(Md, F)
            torch.cuda.synchronize()
            times.append(1e3 * (time.perf_counter() - t0))
            iters.append(tinfo["iterations"])
        J_stop = tplan.objective(Md, F, use_full_k=True)
        tplan.close()
        rec["time_to_tol_ms"] = {
            "tol": TTT_TOL, "p50": float(np.percentile(times, 50)),
            "p99": float(np.percentile(times, 99)), "samples": len(times),
            "percentile_note": "p99 is the largest sample when there are fewer than 100",
            "iterations": int(statistics.median(iters)), "objective_full_k": J_stop,
            "objective_gap": (J_stop - J_ref) / J_ref if J_ref else None,
            "rule": ("||f-x||^2+||f-y||^2+||f-z||^2 and ||dy||^2 relative to ||y||^2"
                     if form == "admm" else "||z-f|| and ||dz|| relative to ||z||")}
        # time to the objective gap and to DFCS: one solve continued block by block
        if J_ref is not None:
            trplan = make_plan(form, prec, max_iter=TRACE_BLOCK, check_every=0)
            trplan.solve(Md, F)                        # warm (plan-time tuning done)
            rec["trace"] = trace_to_tolerance(trplan, Md, F, J_full_of(trplan), f_ref, J_ref,
                                              args.trace_budget, args.ref_iters, stream)
            trplan.close()
            hit = rec["trace"]["gap"][f"{GAP_TOLS[-1]:g}"]
            ttt[(form, prec)] = hit["ms"] if hit else float("inf")
        results[key] = rec
        torch.cuda.empty_cache()

    if args.form == "auto":
        reached = {fp: t for fp, t in ttt.items() if t != float("inf")}
        if reached:
            head = min(reached, key=reached.get)
        else:
            head = ("lowrank", "tf32x3") if ("lowrank", "tf32x3") in available else available[0]
    else:
        head = explicit
    forms_to_run = [head] if args.quick else [head] + [fp for fp in available if fp != head]
    headline = None
    for form, prec in forms_to_run:
        key = form_key(form, prec)
        plan = make_plan(form, prec)
        steps = args.steps if (form, prec) == head else max(2, min(3, args.steps))
        warm = args.warmup if (form, prec) == head else 1
        for _ in range(warm):
            plan.solve_async(Md, F)
        torch.cuda.synchronize()
        plan.profile(True)
        plan.profile_read()
        launches0 = ssm.launch_count()
        clocks = ClockSampler(dist.local)
        dist.barrier()
        torch.cuda.synchronize()
        if (form, prec) == head:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_" + key)
        e0.record(stream)
        for _ in range(steps):
            plan.solve_async(Md, F)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        dist.barrier()
        ms = e0.elapsed_time(e1)
        clk = clocks.stop() if (form, prec) == head else None
        launches = ssm.launch_count() - launches0
        kms, kl = plan.profile_read()
        plan.profile(False)
        ms_max = dist.max(ms)
        per_step = ms_max / steps
        value = weak_value(dist.world, N, Q, per_step / 1e3)
        info = plan.solve(Md, F)[1]
        launch = plan.launch_info()
        rec = results.setdefault(key, {})
        rec.update({"value": value, "ms_per_step": per_step, "launch": launch,
                    "us_per_iteration": 1e3 * per_step / ITERS_PER_STEP,
                    "rank": info["rank"], "gpu_launches": launches,
                    "main_kernel_ms_avg": kms / max(kl, 1), "main_kernel_launches": kl})
        fused = int(launch.get("tc_fused", 0))
        kname, kfile, bound, amount, unit, tkey = dominant_kernel(form, prec, Q, N,
                                                                  info["rank"], fused)
        avg_s = kms / max(kl, 1) / 1e3
        pk = measured_peaks()
        if bound == "hbm":
            peak = pk["hbm_gbs"] if pk else 6800.0
            achieved = amount / avg_s / 1e9
            peak_src = "of measured hbm_gbs" if pk else "of fallback 6.8 TB/s"
        elif bound == "tensor":
            peak = pk["bf16_tflops_sustained"] if pk else 1700.0
            achieved = amount / avg_s / 1e12
            peak_src = "of measured bf16_tflops_sustained" if pk else "of fallback"
        else:
            # FP32 SIMT: 152 SMs x 128 FP32 lanes x 2 flop x max SM clock
            mhz = (pk or {}).get("sm_max_mhz", 2070.0)
            peak = 152 * 128 * 2 * mhz * 1e6 / 1e12
            achieved = amount / avg_s / 1e12
            peak_src = "derived: 152 SM x 128 FP32 lanes x 2 x sm_max_mhz"
        rec["roofline"] = {"bound": bound, "kernel": tkey, "achieved": achieved, "peak": peak,
                           "unit": unit, "frac": achieved / peak, "peak_source": peak_src,
                           "traffic": traffic_record(kfile, tkey),
                           "algorithmic_per_launch": amount}
        if (form, prec) == head:
            headline = {"rec": rec, "clocks": clk, "launches": launches,
                        "roofline": rec["roofline"]}
            # end to end through the C ABI with host buffers (pinned), copies timed
            Mh = torch.from_numpy(M).pin_memory()
            Fh = torch.empty((Q, N), dtype=torch.float32).pin_memory()
            plan.solve_host(Mh, Fh)
            e2e_times = []
            dist.barrier()
            for _ in range(max(2, min(args.steps, 5))):
                t0 = time.perf_counter()
                plan.solve_host(Mh, Fh)
                e2e_times.append(time.perf_counter() - t0)
            e2e_s = dist.max(statistics.median(e2e_times))
            headline["e2e"] = {"value": weak_value(dist.world, N, Q, e2e_s),
                               "unit": METRIC, "h2d_bytes_per_step": int(P * N * 4),
                               "d2h_bytes_per_step": int(Q * N * 4)}
            headline["plan_ms"] = info["plan_ms"]
        plan.close()

    # CPU baseline: the FP64 oracle as it stands, a bounded sample of this workload,
    # and the error of each GPU form after the same iteration count
    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_and_errors(K, M, w, Md, F, make_plan, forms_to_run)

    serving = None
    if dist.world == 1 and not args.no_serving:
        serving = bench_serving(args)
    batching = None
    if dist.world == 1 and not args.no_batching:
        batching = bench_batching()

    workloads = None
    if dist.world == 1 and not args.quick and not args.no_workloads:
        workloads = bench_workloads(args)
        workloads["mrf_b1"] = bench_multidict()

    if dist.rank == 0:
        hl = headline
        htt = hl["rec"].get("time_to_tol_ms", {})
        tr = hl["rec"].get("trace", {})
        dtype = {"fp32": "f32", "bf16x3": "bf16x3+f32", "tf32x3": "tf32x3+f32"}[head[1]]
        out = {
            "metric": METRIC, "value": hl["rec"]["value"], "unit": METRIC,
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": hl["rec"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD}: {describe(w)} "
                                   f"(N={N}), P={P}, Q={Q}, lambda={w.lam}, beta={w.beta:.4g}",
                       "form": form_key(*head), "iters_per_step": ITERS_PER_STEP,
                       "check_every": CHECK_EVERY, "rank": hl["rec"]["rank"],
                       "plan_ms": hl["plan_ms"],
                       "l2": f"inputs larger than L2 (each Q x N state array is "
                             f"{Q * N * 4 / 1e6:.0f} MB)",
                       "parallelism": f"replicas x{dist.world}"},
            "clocks": hl["clocks"], "e2e": hl["e2e"], "gpu_launches": hl["launches"],
            "roofline": hl["roofline"], "cpu_baseline": cpu and cpu["baseline"],
            "time_to_tol_ms": {
                "residual_rule": htt,
                "objective_gap": tr.get("gap"), "dfcs": tr.get("dfcs"),
                "trace_last": tr.get("last"),
                "definition": f"objective_gap: first block of {TRACE_BLOCK} iterations with "
                              "(J - J_ref) / J_ref at or below the tolerance (J with the full "
                              "K); dfcs: ||z - f_ref|| / ||f_ref|| <= "
                              f"{DFCS_TOL:g} (Eq. 33); device time of one solve continued "
                              "block by block"},
            "reference": reference,
            "forms": results,
            "workloads": workloads,
            "err_vs_oracle": cpu and cpu["errors"],
            "serving": serving,
            "batching": batching,
        }
        print(json.dumps(out), flush=True)
    dist.close()


WORKLOAD_LINES = ["rr3d_t1t2", "mrf2d"]


def patch_z(K, M, dims, lam, beta, xi, n_iter, centre, dense, rank):
    """z at `centre` after n_iter iterations from the FP64 oracle run on the box of
    half-width n_iter around it (a voxel's iterate depends only on data within grid
    distance n_iter; xi is the whole grid's, Eq. 32)."""
    from oracle import ladmm as L
    lo = [max(0, c - n_iter) for c in centre]
    hi = [min(d, c + n_iter + 1) for c, d in zip(centre, dims)]
    pd = tuple(h - l for l, h in zip(lo, hi))
    cols = []
    for idx in np.ndindex(*reversed(pd)):
        coord = list(reversed(idx))
        flat, stride = 0, 1
        for ax in range(len(dims)):
            flat += (lo[ax] + coord[ax]) * stride
            stride *= dims[ax]
        cols.append(flat)
    res = L.ladmm(K, M[:, cols], pd, lam, beta, xi_p=xi, rank=rank, dense=dense,
                  iters=n_iter, check_every=0)
    loc, stride, flat, fstride = 0, 1, 0, 1
    for ax in range(len(dims)):
        loc += (centre[ax] - lo[ax]) * stride
        stride *= pd[ax]
        flat += centre[ax] * fstride
        fstride *= dims[ax]
    return res["z"][:, loc], flat


def bench_workloads(args):
    """The 3D T1-T2 (96x96x64, P = 64, Q = 1600) and fingerprinting (192x192, P = 1000,
    Q = 900) workloads: per form, the device time per iteration (difference of two solve
    lengths, CUDA events), the dominant kernel's roofline fraction, and the error at a
    sampled voxel against the FP64 oracle on its patch after a few iterations."""
    import torch

    from oracle import grid
    from paper_2401_12890_gb300 import ssm, synth
    pk = measured_peaks()
    out = {}
    for name in WORKLOAD_LINES:
        w = synth.WORKLOADS[name]
        K, M, _ = synth.make_problem(name)
        Md = torch.from_numpy(M).cuda()
        F = torch.empty((w.Q, w.N), dtype=torch.float32, device="cuda")
        xi = grid.xi_p_rule(w.lam, w.dims)
        centre = tuple(d // 2 for d in w.dims)
        n_err = 4 if len(w.dims) == 3 else 8
        rec = {"dims": list(w.dims), "P": w.P, "Q": w.Q, "N": w.N, "forms": {}}
        for form, prec in [("lowrank", "tf32x3"), ("lowrank", "fp32"), ("dense", "bf16x3"),
                           ("dense", "fp32")]:
            key = form_key(form, prec)
            slow = form == "dense" and prec == "fp32"
            k1, k2 = (2, 6) if slow else (10, 30)
            times = {}
            try:
                plan = ssm.Plan(K, w.dims, w.lam, w.beta, form=form, precision=prec,
                                max_iter=k1, check_every=0)
            except ssm.SsmError as e:
                rec["forms"][key] = {"unsupported": str(e)}
                continue
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for k in (k1, k2):
                plan.set_max_iter(k)
                plan.solve_async(Md, F)
                torch.cuda.synchronize()
                e0.record()
                plan.solve_async(Md, F)
                e1.record()
                torch.cuda.synchronize()
                times[k] = e0.elapsed_time(e1)
            per_it = (times[k2] - times[k1]) / (k2 - k1)
            plan.set_max_iter(k2)
            plan.profile(True)
            plan.solve_async(Md, F)
            kms, kl = plan.profile_read()
            plan.profile(False)
            info = plan.info()
            launch = plan.launch_info()
            _, kfile, bound, amount, unit, tkey = dominant_kernel(
                form, prec, w.Q, w.N, info["rank"], int(launch.get("tc_fused", 0)))
            avg_s = kms / max(kl, 1) / 1e3
            if bound == "hbm":
                peak = pk["hbm_gbs"] if pk else 6800.0
                achieved = amount / avg_s / 1e9
            elif bound == "tensor":
                peak = pk["bf16_tflops_sustained"] if pk else 1700.0
                achieved = amount / avg_s / 1e12
            else:
                peak = 152 * 128 * 2 * (pk or {}).get("sm_max_mhz", 2070.0) * 1e6 / 1e12
                achieved = amount / avg_s / 1e12
            plan.set_max_iter(n_err)
            Fz, _ = plan.solve(Md, F)
            zg = Fz.cpu().numpy().astype(np.float64)
            plan.close()
            zr, flat = patch_z(K, M.astype(np.float64), w.dims, w.lam, w.beta, xi, n_err,
                               centre, form == "dense", info["rank"] if form == "lowrank"
                               else None)
            err = float(np.linalg.norm(zg[:, flat] - zr) / max(np.linalg.norm(zr), 1e-300))
            rec["forms"][key] = {
                "us_per_iteration": 1e3 * per_it,
                "value": w.N * w.Q / (per_it / 1e3), "unit": METRIC, "rank": info["rank"],
                "roofline": {"bound": bound, "kernel": tkey, "achieved": achieved,
                             "peak": peak, "unit": unit, "frac": achieved / peak,
                             "main_kernel_ms_avg": kms / max(kl, 1),
                             "traffic": traffic_record(kfile, tkey, name)},
                "err_vs_oracle": {"voxel": list(centre), "iterations": n_err,
                                  "rel_l2": err, "oracle": "FP64 on the voxel's patch"}}
            torch.cuda.empty_cache()
        out[name] = rec
        del Md, F
        torch.cuda.empty_cache()
    return out


def patch_z_multi(Ks, labels, M, dims, lam, beta, xi, n_iter, centre):
    """As patch_z for spatially varying dictionaries (oracle.multidict), with only the
    patch's dictionaries (relabelling them changes nothing)."""
    from oracle import multidict as MD
    lo = [max(0, c - n_iter) for c in centre]
    hi = [min(d, c + n_iter + 1) for c, d in zip(centre, dims)]
    pd = tuple(h - l for l, h in zip(lo, hi))
    cols = []
    for idx in np.ndindex(*reversed(pd)):
        coord = list(reversed(idx))
        flat, stride = 0, 1
        for ax in range(len(dims)):
            flat += (lo[ax] + coord[ax]) * stride
            stride *= dims[ax]
        cols.append(flat)
    present, local = np.unique(labels[cols], return_inverse=True)
    res = MD.ladmm_multi([Ks[c] for c in present], local, M[:, cols], pd, lam, beta, xi_p=xi,
                         iters=n_iter, check_every=0)
    loc, stride, flat, fstride = 0, 1, 0, 1
    for ax in range(len(dims)):
        loc += (centre[ax] - lo[ax]) * stride
        stride *= pd[ax]
        flat += centre[ax] * fstride
        fstride *= dims[ax]
    return res["z"][:, loc], flat


def bench_multidict():
    """The fingerprinting stand-in with a dictionary per B1 level (61 levels, 156 x 156,
    P = 120, Q = 900): device time per iteration of the spatially varying dictionary path
    (difference of two solve lengths, CUDA events), its kernel's roofline fraction, the
    same grid with one dictionary for every voxel (the single-dictionary FP32 low-rank
    kernel) for the cost of the per-voxel dictionaries, and the error at sampled voxels
    against the FP64 oracle on their patches."""
    import torch

    from oracle import grid
    from paper_2401_12890_gb300 import ssm, synth
    pk = measured_peaks()
    w = synth.B1_WORKLOAD
    Ks, labels, M, _ = synth.make_b1_problem()
    Md = torch.from_numpy(M).cuda()
    F = torch.empty((w.Q, w.N), dtype=torch.float32, device="cuda")
    rec = {"dims": list(w.dims), "P": w.P, "Q": w.Q, "N": w.N, "levels": len(Ks),
           "labels": "a smooth B1 field quantised to the levels"}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def per_iteration(plan, k1=20, k2=60):
        times = {}
        for k in (k1, k2):
            plan.set_max_iter(k)
            plan.solve_async(Md, F)
            torch.cuda.synchronize()
            e0.record()
            plan.solve_async(Md, F)
            e1.record()
            torch.cuda.synchronize()
            times[k] = e0.elapsed_time(e1)
        return (times[k2] - times[k1]) / (k2 - k1)

    t0 = time.perf_counter()
    plan = ssm.MultiPlan(Ks, labels, w.dims, w.lam, w.beta, max_iter=20, check_every=0)
    plan_s = time.perf_counter() - t0
    per_it = per_iteration(plan)
    plan.set_max_iter(60)
    plan.profile(True)
    plan.solve_async(Md, F)
    kms, kl = plan.profile_read()
    plan.profile(False)
    info = plan.info()
    launch = plan.launch_info()
    r = info["rank"]
    amount = 8.0 * w.Q * w.N + 12.0 * r * w.N + 4.0 * w.N
    avg_s = kms / max(kl, 1) / 1e3
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = amount / avg_s / 1e9
    n_err = 6
    plan.set_max_iter(n_err)
    Fz, _ = plan.solve(Md, F)
    zg = Fz.cpu().numpy().astype(np.float64)
    plan.close()
    xi = grid.xi_p_rule(w.lam, w.dims)
    errs = []
    for centre in [(w.dims[0] // 2, w.dims[1] // 2), (0, 0), (w.dims[0] - 1, 17)]:
        zr, flat = patch_z_multi(Ks, labels, M.astype(np.float64), w.dims, w.lam, w.beta, xi,
                                 n_err, centre)
        errs.append(float(np.linalg.norm(zg[:, flat] - zr) / max(np.linalg.norm(zr), 1e-300)))
    rec["lowrank_fp32_multi"] = {
        "us_per_iteration": 1e3 * per_it, "value": w.N * w.Q / (per_it / 1e3), "unit": METRIC,
        "rank": r, "plan_s": plan_s, "segments_grid": launch.get("lowrank_grid"),
        "roofline": {"bound": "hbm", "kernel": "table_iter_kernel", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "main_kernel_ms_avg": kms / max(kl, 1),
                     "algorithmic_per_launch": amount,
                     "traffic": traffic_record("ssm_table.cu", "table_iter_kernel",
                                               w.name)},
        "err_vs_oracle": {"voxels": 3, "iterations": n_err, "max_rel_l2": max(errs),
                          "oracle": "FP64 oracle.multidict on each voxel's patch"}}
    # the same grid and data with one dictionary (the centre voxel's) for every voxel
    c = int(labels[(w.dims[1] // 2) * w.dims[0] + w.dims[0] // 2])
    one = ssm.Plan(Ks[c], w.dims, w.lam, w.beta, form="lowrank", precision="fp32",
                   max_iter=20, check_every=0)
    per_one = per_iteration(one)
    one.close()
    rec["lowrank_fp32_one_dictionary"] = {
        "us_per_iteration": 1e3 * per_one, "value": w.N * w.Q / (per_one / 1e3),
        "unit": METRIC, "note": "the centre voxel's dictionary for every voxel: the cost of "
                                "one dictionary per voxel is the ratio of the two lines"}
    del Md, F
    torch.cuda.empty_cache()
    return rec


def cpu_baseline_and_errors(K, M, w, Md, F, make_plan, forms):
    """The FP64 oracle as it stands (the low-rank Algorithm 2, the same form as the
    TF32x3 and FP32 low-rank lines) on the host cores: the rate of its iterations (a run
    of 4 iterations minus a run of 1, so the setup -- SVD, projections -- cancels), and
    each GPU form's error against it after 3 iterations."""
    from oracle import ladmm as L
    iters = 3
    t0 = time.perf_counter()
    L.ladmm(K, M, w.dims, w.lam, w.beta, iters=1, check_every=0)
    t1 = time.perf_counter()
    ref = L.ladmm(K, M, w.dims, w.lam, w.beta, iters=1 + iters, check_every=0)
    t2 = time.perf_counter()
    dt = max((t2 - t1) - (t1 - t0), 1e-9)
    ref = L.ladmm(K, M, w.dims, w.lam, w.beta, iters=iters, check_every=0)
    baseline = {"value": w.N * w.Q * iters / dt, "unit": METRIC, "cores": os.cpu_count(),
                "kind": "oracle",
                "sample": f"FP64 numpy oracle, low-rank Algorithm 2 (r={ref['r']}), full "
                          f"{WORKLOAD} inputs: {iters} iterations timed as the difference of "
                          f"a {1 + iters}-iteration and a 1-iteration run ({dt:.1f} s); "
                          "numpy's default BLAS threading"}
    errors = {}
    refd = refa = None
    for form, prec in forms:
        if form == "dense" and refd is None:
            refd = L.ladmm(K, M, w.dims, w.lam, w.beta, dense=True, iters=iters, check_every=0)
        if form == "admm" and refa is None:
            from oracle import admm as A
            refa = A.admm(K, M, w.dims, w.lam, w.beta, iters=iters)
        pl = make_plan(form, prec, max_iter=iters, check_every=0)
        out, _ = pl.solve(Md, F)
        z = out.cpu().numpy().astype(np.float64)
        pl.close()
        zr = refa["y"] if form == "admm" else (refd if form == "dense" else ref)["z"]
        errors[form_key(form, prec)] = {
            "iterations": iters,
            "rel_fro": float(np.linalg.norm(z - zr) / np.linalg.norm(zr))}
    return {"baseline": baseline, "errors": errors}



# --------------------------------------------------------------------------------------
# serving: Poisson-arriving solves of mixed shapes through the continuous-batching server
# --------------------------------------------------------------------------------------
SERVE_SHAPES = ["dr2d_tiny", "dr2d_slice", "rr3d_t1t2"]
# (form, precision, group_small): the last runs the FP32 low-rank form with the small
# requests solved in groups of up to 16
SERVE_FORMS = [("lowrank", "tf32x3", 0), ("dense", "bf16x3", 0), ("lowrank", "fp32", 16)]
SERVE_SEED = 46


def bench_serving(args):
    """64 requests, shapes drawn uniformly from the tiny 2D, 2D slice and 3D T1-T2
    workloads (seed 46), arriving as a Poisson process at `serve_load` of the measured
    capacity; each request is a fixed budget of `serve_iters` iterations on host
    buffers (M in, F out) through ssm_server_submit / ssm_server_wait. Returns the
    latency percentiles and the aggregate throughput per form."""
    import threading

    import torch

    from paper_2401_12890_gb300 import ssm, synth
    rng = np.random.default_rng(SERVE_SEED)
    kinds = rng.integers(0, len(SERVE_SHAPES), size=args.serve_requests)
    data = {}
    for name in SERVE_SHAPES:
        w = synth.WORKLOADS[name]
        K = synth.dictionary_for(name)
        Ms = [torch.from_numpy(np.ascontiguousarray(
            synth.make_problem(name, seed=w.seed + 100 * j)[1])).cuda() for j in range(2)]
        data[name] = (w, K, Ms)
    iters = args.serve_iters
    out = {"requests": int(args.serve_requests), "iters_per_request": iters,
           "mix": {n: int((kinds == i).sum()) for i, n in enumerate(SERVE_SHAPES)},
           "shapes": {n: {"dims": list(data[n][0].dims), "P": data[n][0].P, "Q": data[n][0].Q}
                      for n in SERVE_SHAPES},
           "arrivals": f"Poisson (seed {SERVE_SEED}), rate = {args.serve_load:g} x capacity, "
                       "capacity = 1 / mean solo service time of the mix",
           "io": "device buffers: M resident on the device, F written to a fresh device "
                 "buffer per request (ssm_server_submit_device)",
           "forms": {}}
    for form, prec, group in SERVE_FORMS:
        key = form_key(form, prec) + ("_grouped" if group else "")
        kw = dict(form=form, precision=prec, max_iter=iters, check_every=0)
        free, _ = torch.cuda.mem_get_info()
        # plans get 60 % of the free memory; the rest holds the requests' F buffers
        with ssm.Server(max_active=4, use_graphs=True, cache_plans=True,
                        hbm_budget=int(0.6 * free), group_small=group) as srv:
            # solo service time per shape (plans built and cached here, as a server
            # running before the measurement would have them)
            solo = {}
            for name in SERVE_SHAPES:
                w, K, Ms = data[name]
                times = []
                for j in range(2):
                    t = srv.submit(K, Ms[j], w.dims, w.lam, w.beta, **kw)
                    times.append(srv.wait(t)[1]["latency_ms"])
                solo[name] = times[-1]
            mean_s = sum(solo[SERVE_SHAPES[k]] for k in kinds) / len(kinds) / 1e3
            rate = args.serve_load / mean_s
            gaps = rng.exponential(1.0 / rate, size=len(kinds))
            arrivals = np.cumsum(gaps) - gaps[0]
            s0 = srv.stats()
            tickets = [None] * len(kinds)
            t0 = time.perf_counter()

            def submitter():
                for i, k in enumerate(kinds):
                    delay = t0 + arrivals[i] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                    w, K, Ms = data[SERVE_SHAPES[k]]
                    tickets[i] = srv.submit(K, Ms[i % 2], w.dims, w.lam, w.beta, **kw)

            th = threading.Thread(target=submitter)
            th.start()
            infos = []
            for i in range(len(kinds)):
                while tickets[i] is None:
                    time.sleep(1e-4)
                infos.append(srv.wait(tickets[i])[1])
            th.join()
            makespan = time.perf_counter() - t0
            st = srv.stats()
        lat = np.array([i["latency_ms"] for i in infos])
        que = np.array([i["queue_ms"] for i in infos])
        work = sum(data[SERVE_SHAPES[k]][0].N * data[SERVE_SHAPES[k]][0].Q * iters for k in kinds)
        per_shape = {}
        for i, name in enumerate(SERVE_SHAPES):
            sel = lat[kinds == i]
            if len(sel):
                per_shape[name] = {"p50": float(np.percentile(sel, 50)),
                                   "p99": float(np.percentile(sel, 99)),
                                   "solo_ms": solo[name]}
        out["forms"][key] = {
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)), "mean": float(lat.mean())},
            "queue_ms": {"p50": float(np.percentile(que, 50)),
                         "p99": float(np.percentile(que, 99))},
            "per_shape_latency_ms": per_shape,
            "throughput": work / makespan, "unit": METRIC,
            "requests_per_s": len(kinds) / makespan, "makespan_s": makespan,
            "arrival_rate_per_s": rate,
            "statuses_ok": int(sum(i["status"] in (ssm.SSM_OK, ssm.SSM_ENOTCONVERGED)
                                   for i in infos)),
            "plans_created": st["plans_created"] - s0["plans_created"],
            "plans_reused": st["plans_reused"] - s0["plans_reused"],
            "peak_hbm_reserved_gb": st["peak_bytes_held"] / 1e9,
            "hbm_budget_gb": st["budget"] / 1e9,
            "launch": "stream priority by footprint class (<= 64 MiB highest, one level per "
                      "factor 4 above); above the first class, persistent kernels in 8 "
                      "launch waves; one of the 4 workers reserved for the first class" +
                      (f"; first-class requests solved in groups of up to {group}"
                       if group else ""),
            "group_sizes": sorted({int(i["group_size"]) for i in infos}),
        }
        torch.cuda.empty_cache()
    return out

# --------------------------------------------------------------------------------------
# batching: many small slices sharing a dictionary, one plan for all of them
# --------------------------------------------------------------------------------------
BATCH_SLICES = 64


def bench_batching():
    """64 slices of the 32 x 32 diffusion-relaxation workload (P = 30, Q = 225), 300
    iterations each: 64 solves in turn on one plan, against one batched plan
    (ssm_plan_batched) solving all slices in the same launches."""
    import torch

    from paper_2401_12890_gb300 import ssm, synth
    w = synth.WORKLOADS["dr2d_tiny"]
    K = synth.dictionary_for("dr2d_tiny")
    Ms = [synth.make_problem("dr2d_tiny", seed=w.seed + 10 * b)[1] for b in range(BATCH_SLICES)]
    Mall = torch.from_numpy(np.ascontiguousarray(np.concatenate(Ms, axis=1))).cuda()
    Md = [torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in Ms]
    work = BATCH_SLICES * w.N * w.Q * w.iters
    out = {"slices": BATCH_SLICES, "slice": f"{w.dims[0]}x{w.dims[1]}, P={w.P}, Q={w.Q}",
           "iterations": w.iters, "unit": METRIC, "forms": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for form, prec in (("lowrank", "tf32x3"), ("lowrank", "fp32"), ("dense", "bf16x3")):
        kw = dict(form=form, precision=prec, max_iter=w.iters, check_every=0)
        one = ssm.Plan(K, w.dims, w.lam, w.beta, **kw)
        one.set_graphs(True)
        F1 = torch.empty((w.Q, w.N), dtype=torch.float32, device="cuda")
        for m in Md[:2]:
            one.solve_async(m, F1)
        torch.cuda.synchronize()
        e0.record()
        for m in Md:
            one.solve_async(m, F1)
        e1.record()
        torch.cuda.synchronize()
        t_seq = e0.elapsed_time(e1) / 1e3
        one.close()
        bat = ssm.Plan(K, w.dims, w.lam, w.beta, batch=BATCH_SLICES, **kw)
        bat.set_graphs(True)
        FB = torch.empty((w.Q, w.N * BATCH_SLICES), dtype=torch.float32, device="cuda")
        for _ in range(2):
            bat.solve_async(Mall, FB)
        torch.cuda.synchronize()
        e0.record()
        bat.solve_async(Mall, FB)
        e1.record()
        torch.cuda.synchronize()
        t_bat = e0.elapsed_time(e1) / 1e3
        bat.close()
        out["forms"][form_key(form, prec)] = {
            "one_by_one_s": t_seq, "batched_s": t_bat, "speedup": t_seq / t_bat,
            "one_by_one_value": work / t_seq, "batched_value": work / t_bat}
    out["heterogeneous_group"] = bench_group()
    return out


GROUP_SHAPES = [((32, 32), 30, 225), ((24, 20), 16, 100), ((48, 16), 24, 64), ((64,), 12, 50),
                ((12, 10, 6), 20, 80), ((40, 40), 30, 144)]


def bench_group(nprob=64, iters=300):
    """64 small problems of six shapes (differing N, P, Q; seed 51), 300 iterations each
    (the low-rank FP32 form): solved one after another (ssm_solve, CUDA graphs) against
    one group (ssm_group_*: one launch per iteration for all of them)."""
    import torch

    from paper_2401_12890_gb300 import ssm, synth
    rng = np.random.default_rng(51)
    kinds = rng.integers(0, len(GROUP_SHAPES), size=nprob)
    plans, Ms, Fs, work = [], [], [], 0
    for i, k in enumerate(kinds):
        dims, P, Q = GROUP_SHAPES[k]
        K, M, _ = synth.random_problem(P, Q, dims, seed=1000 + i, snr=60.0)
        pl = ssm.Plan(K, dims, 0.02, 0.3, form="lowrank", precision="fp32", max_iter=iters,
                      check_every=0)
        pl.set_graphs(True)
        plans.append(pl)
        Ms.append(torch.from_numpy(np.ascontiguousarray(M, np.float32)).cuda())
        Fs.append(torch.empty((Q, pl.N), dtype=torch.float32, device="cuda"))
        work += pl.N * Q * iters
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for pl, M, F in zip(plans, Ms, Fs):
        pl.solve_async(M, F)
    torch.cuda.synchronize()
    e0.record()
    for pl, M, F in zip(plans, Ms, Fs):
        pl.solve_async(M, F)
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    grp = ssm.Group(plans)
    grp.solve(Ms, Fs)
    torch.cuda.synchronize()
    n0 = ssm.launch_count()
    e0.record()
    grp.solve(Ms, Fs)
    e1.record()
    torch.cuda.synchronize()
    t_grp = e0.elapsed_time(e1) / 1e3
    launches = ssm.launch_count() - n0
    grp.close()
    for pl in plans:
        pl.close()
    return {"problems": nprob, "iterations": iters,
            "shapes": [{"dims": list(d), "P": P, "Q": Q} for d, P, Q in GROUP_SHAPES],
            "mix": [int((kinds == j).sum()) for j in range(len(GROUP_SHAPES))],
            "one_by_one_s": t_seq, "group_s": t_grp, "speedup": t_seq / t_grp,
            "one_by_one_value": work / t_seq, "group_value": work / t_grp, "unit": METRIC,
            "group_launches": launches}


# --------------------------------------------------------------------------------------
# reference arm: the FP64 oracle itself on the host cores
# --------------------------------------------------------------------------------------
def bench_reference(args):
    world, rank, _ = dist_env()
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group(backend="gloo")
        if rank != 0:
            tdist.destroy_process_group()
            return
    from oracle import ladmm as L
    from paper_2401_12890_gb300 import synth
    w = synth.WORKLOADS[WORKLOAD]
    K, M, _ = synth.make_problem(WORKLOAD)
    # a step: 2 iterations of the low-rank Algorithm 2, continuing from the previous
    # step's state (z, d) -- the oracle forms its factors and projections anew per call
    iters = 2
    z = d = None
    for _ in range(args.warmup):
        res = L.ladmm(K, M, w.dims, w.lam, w.beta, iters=iters, check_every=0, z0=z, d0=d)
        z, d = res["z"], res["d"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = L.ladmm(K, M, w.dims, w.lam, w.beta, iters=iters, check_every=0, z0=z, d0=d)
        z, d = res["z"], res["d"]
    dt = time.perf_counter() - t0
    value = w.N * w.Q * iters * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: {describe(w)} "
                               f"(N={w.N}), P={w.P}, Q={w.Q}, lambda={w.lam}",
                   "form": "lowrank (Algorithm 2) FP64 oracle"},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": f"each step: {iters} iterations of the oracle on the full "
                                   "workload, continuing the previous step's state (setup: "
                                   "SVD and projections, formed anew in every step)"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


def main():
    global WORKLOAD
    args = parse_args()
    WORKLOAD = args.workload
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
