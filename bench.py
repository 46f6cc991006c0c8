"""Throughput benchmark: |M|^2 points/s of e- gamma -> e- + k gamma on B300.

Default workload: e- gamma -> e- + 4 gamma (120 diagrams), 1,048,576 seeded
RAMBO points at omega = 4 m_e, all 128 helicity/polarisation states summed.
One step = one evaluation of the whole batch.  The FP32-mixed path gives the
line's value; the plain FP64 path is timed the same way and reported beside
it, each with its roofline against the FMA-pipe peak.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl ours|reference]

Under torchrun every rank evaluates its own batch (weak scaling) and rank 0
prints one JSON line.  --impl reference times the CPU oracle on the host
cores instead (a bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_19456_b300 import phasespace as ps  # noqa: E402

SM_COUNT = 148
SM_MAX_MHZ = 2032.0
FP32_LANES_PER_SM = 128
# Peaks of the FMA pipes from unit counts and the maximum SM clock:
# FP32 148 SMs x 128 lanes x 2 FLOP x 2.032 GHz; FP64 the nominal B300 rate.
PEAK_FP32_TFLOPS = SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
PEAK_FP64_TFLOPS = 1.25
# Version of the forward kernels (arithmetic, shared-memory layout, launch
# shape); bumped with every change to them.  DRAM traffic recorded in
# profiles/traffic.json is reported only for the version it was measured on.
# FWD: the table-driven kernel (qed_fwd.cu); SPEC: the straight-line
# specialised kernel (the kernel version its generator writes).
FWD_KERNEL_VERSION = "fwd-9"
SPEC_KERNEL_VERSION = "spec-6"
# Mixed-precision and FP64 per-point bounds against the oracle (as the GPU
# tests state them): 64 u32 max(kappa, 1) and max(1e-12, 64 u64 kappa).
U32, U64 = 2.0 ** -24, 2.0 ** -53
C_MIX = 64
# The same for the kernel of the distributively rewritten DAG.
RW_KERNEL_VERSION = "rw-5"


def recorded_traffic(workload: str, prec: str, n_points: int, dag: str = "plain", form: str = "table"):
    if dag != "plain":
        key, version = f"{workload}/{dag}/{prec}", RW_KERNEL_VERSION
    elif form == "specialised":
        key, version = f"{workload}/specialised/{prec}", SPEC_KERNEL_VERSION
    else:
        key, version = f"{workload}/{prec}", FWD_KERNEL_VERSION
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("kernel_version") != version or rec.get("n_points") != n_points:
        return None
    return rec["bytes_per_launch"]


def host_chunks(n: int) -> list:
    """Chunk sizes of one qed_eval_host call on n points (one kernel launch
    each): starting at an eighth of the largest chunk, doubling up to it."""
    chunk = min(n, max(1 << 16, (n + 7) // 8))
    size, off, out = max(min(chunk, 8192), chunk // 8), 0, []
    while off < n:
        m = min(size, n - off)
        out.append(m)
        off += m
        size = min(chunk, 2 * size)
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during a timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        if not getattr(self, "lines", None):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(mom: np.ndarray, k: int, target_cpu_s: float = 15.0):
    """The oracle, as it stands, on the host cores: batches of the workload's
    points until about target_cpu_s of CPU time (wall x threads) is spent.
    Also returns the oracle's |M|^2 and kappa on those points (sample
    indices cores .. cores + done), against which the GPU results of the same
    points are compared."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.m2(mom[:cores], threads=cores)  # thread pool start-up
    done, off, t_wall = 0, cores, 0.0
    batch = cores
    refs, kaps = [], []
    while t_wall * cores < target_cpu_s and off + batch <= len(mom):
        t0 = time.perf_counter()
        r, kp = oracle.m2(mom[off:off + batch], threads=cores, kappa=True)
        dt = time.perf_counter() - t0
        refs.append(r)
        kaps.append(kp)
        t_wall += dt
        done += batch
        off += batch
        if dt < 0.5:
            batch *= 2
    # the same oracle on one thread (the paper times single-threaded code)
    b1, t1, off1 = max(1, batch // cores), 0.0, off
    done1 = 0
    while t1 < 3.0 and off1 + b1 <= len(mom):
        t0 = time.perf_counter()
        oracle.m2(mom[off1:off1 + b1], threads=1)
        t1 += time.perf_counter() - t0
        done1 += b1
        off1 += b1
    line = {"value": done / t_wall, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} of the {len(mom)} k={k} points (all states summed), "
                      f"{t_wall:.1f} s wall on {cores} threads",
            "single_thread_points_per_s": done1 / t1 if t1 > 0 else None}
    sample = (np.arange(cores, cores + done), np.concatenate(refs), np.concatenate(kaps)) if refs else None
    return line, sample


def error_stats(got, ref, kap, prec):
    """Relative error of GPU results against the oracle, with the per-point
    bound of the tests (max_over_bound <= 1: every point within it)."""
    rel = np.abs(np.asarray(got) / ref - 1.0)
    if prec == "mixed":
        bound, text = C_MIX * U32 * np.maximum(kap, 1.0), "64 u32 max(kappa, 1)"
    else:
        bound, text = np.maximum(1e-12, 64 * U64 * kap), "max(1e-12, 64 u64 kappa)"
    return {"n": int(rel.size), "median": float(np.median(rel)), "max": float(rel.max()),
            "kappa_max": float(np.max(kap)), "max_over_bound": float(np.max(rel / bound)), "bound": text}


def measure_peaks(local):
    """FMA-pipe peaks of this GPU, measured in this run (the roofline
    denominators), with the SM clocks sampled while they run."""
    from paper_2511_19456_b300 import measure_fma_peak
    with ClockSampler(local) as cs:
        fp32 = measure_fma_peak("mixed")
        fp64 = measure_fma_peak("fp64")
    return {"fp32_tflops": fp32, "fp64_tflops": fp64, "clocks": cs.summary(),
            "how": "independent FMA chains on every SM, CUDA events; FP32 the larger of scalar and "
                   "packed (two per instruction) chains"}


def run_reference(args, workload):
    """--impl reference: the FP64 oracle on the host cores, one bounded sample per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = ps.WORKLOADS[workload]
    cores = os.cpu_count() or 1
    per_step = max(cores, 4 * cores)
    mom = ps.points(w["k"], per_step * (args.steps + args.warmup), w["omega"], w["seed"])
    steps = []
    for s in range(args.warmup + args.steps):
        chunk = mom[s * per_step:(s + 1) * per_step]
        t0 = time.perf_counter()
        oracle.m2(chunk, threads=cores)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            steps.append(dt)
    t = sum(steps)
    value = per_step * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload, "dag": "plain", "k": w["k"], "n_points": w["n_points"],
                   "omega": w["omega"], "states_summed": 2 ** (w["k"] + 3) if w["summed"] else 1,
                   "sample_points_per_step": per_step,
                   "note": "each step a bounded sample of the workload on the host cores"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} points per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


METRIC = "|M|^2 points/s on 1 B300 (e gamma -> e + k gamma), FP32-mixed vs FP64, % of FLOP peak"


def time_calls(fn, steps, warmup):
    """CUDA-event time per call of fn() on the current stream (ms)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_other(args):
    """Measurement lines for the configurations other than the headline one.

    compton_k6_fixed: FP64 and mixed forward, FP64 adjoint (qed_eval_grad).
    compton_k7: mixed forward and adjoint on the full 131,072 points; the FP64
      forward on a --fp64-points slice (one FP64 step of the full set takes
      about 170 s).
    batched: 64 requests, k = 1..5; the tuned graph launch (mixed and FP64)
      against one launch per request (the plain FP64 GPU path).
    """
    import torch
    from paper_2511_19456_b300 import Batch, Plan
    torch.cuda.set_device(0)
    res = {"workload": args.workload, "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    if args.workload == "batched":
        reqs = ps.batched_requests()
        moms = [torch.from_numpy(ps.points(r["k"], r["n_points"], r["omega"], r["seed"])).cuda()
                for r in reqs]
        n_tot = sum(r["n_points"] for r in reqs)
        for prec in ("mixed", "fp64"):
            plans = {k: Plan(k, precision=prec) for k in range(1, 6)}
            flops = sum(plans[r["k"]].info()["flops_per_point"] * r["n_points"] for r in reqs)
            batch = Batch([plans[r["k"]] for r in reqs], [r["n_points"] for r in reqs])
            outs = batch.outputs()
            tuned_ms = batch.tune(moms, outs) if prec == "mixed" else None
            steps = args.steps if prec == "mixed" else 1
            ms_b = time_calls(lambda: batch.eval(moms, outs), steps, 1)
            seq_outs = [torch.empty_like(o) for o in outs]

            def seq():
                for r, m, o in zip(reqs, moms, seq_outs):
                    plans[r["k"]].eval(m, o)
            ms_s = time_calls(seq, steps, 1)
            same = all(torch.equal(a, b) for a, b in zip(outs, seq_outs))
            peak = PEAK_FP32_TFLOPS if prec == "mixed" else PEAK_FP64_TFLOPS
            res[prec] = {"batched_points_per_s": n_tot / (ms_b * 1e-3), "batched_ms": ms_b,
                         "sequential_points_per_s": n_tot / (ms_s * 1e-3), "sequential_ms": ms_s,
                         "launches_sequential": len(reqs), "launches_batched": 1,
                         "batched_tflops": flops / (ms_b * 1e-3) / 1e12,
                         "batched_frac_of_peak": flops / (ms_b * 1e-3) / 1e12 / peak,
                         "tune_best_ms": tuned_ms, "batch_info": batch.info(),
                         "identical_to_sequential": same}
        res.update(metric=METRIC, unit="points/s", value=res["mixed"]["batched_points_per_s"],
                   config={"workload": "batched", "requests": len(reqs), "n_points": n_tot,
                           "k": "1..5", "omega": "U[1,8]", "states": "summed"},
                   speedup_batched_mixed_vs_sequential_fp64=res["fp64"]["sequential_ms"] / res["mixed"]["batched_ms"],
                   speedup_batched_fp64_vs_sequential_fp64=res["fp64"]["sequential_ms"] / res["fp64"]["batched_ms"])
        print(json.dumps(res), flush=True)
        return
    w = ps.WORKLOADS[args.workload]
    k, n = w["k"], (args.n_points or w["n_points"])
    hel = None if w["summed"] else w["hel"]
    mom = torch.from_numpy(ps.points(k, n, w["omega"], w["seed"])).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    grad = torch.empty((n, k, 3), dtype=torch.float64, device="cuda")
    for prec in ("mixed", "fp64"):
        plan = Plan(k, summed=w["summed"], hel=hel, precision=prec)
        info = plan.info()
        nn = n if prec == "mixed" or args.fp64_points is None else min(n, args.fp64_points)
        mm, oo, gg = mom[:nn], out[:nn], grad[:nn]
        ms_f = time_calls(lambda: plan.eval(mm, oo), args.steps, args.warmup)
        peak = PEAK_FP32_TFLOPS if prec == "mixed" else PEAK_FP64_TFLOPS
        leg = {"n_points": nn, "forward_points_per_s": nn / (ms_f * 1e-3), "forward_ms": ms_f,
               "forward_tflops": info["flops_per_point"] * nn / (ms_f * 1e-3) / 1e12,
               "forward_frac_of_peak": info["flops_per_point"] * nn / (ms_f * 1e-3) / 1e12 / peak}
        try:
            ms_g = time_calls(lambda: plan.eval_grad(mm, oo, gg), args.steps, args.warmup)
            leg.update(adjoint_points_per_s=nn / (ms_g * 1e-3), adjoint_ms=ms_g,
                       adjoint_over_forward_time=ms_g / ms_f)
        except Exception as exc:  # plan without an adjoint in this precision
            leg.update(adjoint=str(exc))
        res[prec] = leg
    res.update(metric=METRIC, unit="points/s", value=res["mixed"]["forward_points_per_s"],
               config={"workload": args.workload, "k": k, "n_points": n, "omega": w["omega"],
                       "states": "summed" if w["summed"] else "fixed"},
               speedup_mixed_vs_fp64=res["mixed"]["forward_points_per_s"] / res["fp64"]["forward_points_per_s"])
    print(json.dumps(res), flush=True)


def run_rewrite_compare(args):
    """The distributively rewritten DAG against the plain (node-reduced) DAG,
    forward pass, both precisions, on the headline workloads.  For each leg:
    points/s of both DAGs on the same points, the speed-up, and the largest
    relative difference between them.  The plain FP64 pass at k = 7 runs on a
    slice (one full step takes minutes)."""
    import torch
    from paper_2511_19456_b300 import Plan
    torch.cuda.set_device(0)
    res = {"workload": "rewrite_vs_plain", "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
           "metric": METRIC, "unit": "points/s"}
    slices = {"compton_k4": (None, None), "compton_k6_fixed": (None, 16384), "compton_k7": (16384, 2048)}
    for wname, (n_mixed, n_fp64) in slices.items():
        w = ps.WORKLOADS[wname]
        k = w["k"]
        hel = None if w["summed"] else w["hel"]
        mom_all = torch.from_numpy(ps.points(k, w["n_points"], w["omega"], w["seed"])).cuda()
        legs = {}
        for prec, n_cut in (("mixed", n_mixed), ("fp64", n_fp64)):
            n = w["n_points"] if n_cut is None else n_cut
            mom = mom_all[:n]
            leg = {"n_points": n}
            outs = {}
            for dag in ("rewrite", "plain"):
                plan = Plan(k, summed=w["summed"], hel=hel, precision=prec, rewrite=(dag == "rewrite"))
                out = torch.empty(n, dtype=torch.float64, device="cuda")
                steps = args.steps if dag == "rewrite" else max(1, min(args.steps, 3))
                ms = time_calls(lambda: plan.eval(mom, out), steps, 1 if dag == "plain" else args.warmup)
                leg[dag] = {"ms": ms, "points_per_s": n / (ms * 1e-3),
                            "flops_per_point": plan.info()["flops_per_point"]}
                outs[dag] = out
            leg["speedup_rewrite_vs_plain"] = leg["plain"]["ms"] / leg["rewrite"]["ms"]
            leg["max_rel_diff"] = float(((outs["rewrite"] / outs["plain"]) - 1).abs().max())
            legs[prec] = leg
        # the full workload through the rewrite: the headline rate of this DAG
        for prec in ("mixed", "fp64"):
            plan = Plan(k, summed=w["summed"], hel=hel, precision=prec, rewrite=True)
            out = torch.empty(w["n_points"], dtype=torch.float64, device="cuda")
            ms = time_calls(lambda: plan.eval(mom_all, out), args.steps, args.warmup)
            legs[prec]["rewrite_full_points_per_s"] = w["n_points"] / (ms * 1e-3)
        res[wname] = legs
    res["value"] = res["compton_k4"]["mixed"]["rewrite_full_points_per_s"]
    res["config"] = {"workload": "rewrite_vs_plain", "k": "4 (summed), 6 (fixed), 7 (summed)"}
    print(json.dumps(res), flush=True)


def run_cross_section(args):
    """Monte Carlo total cross sections (qed_cross_section): the points are
    generated on the device (seeded RAMBO, weights), evaluated and reduced on
    the device, one synchronous call per step.  k = 1 in FP64 against the
    closed-form Klein-Nishina cross section (e = m = 1), k = 4 in mixed
    precision; points/s of the whole call."""
    import torch
    from paper_2511_19456_b300 import Plan, cross_section
    torch.cuda.set_device(0)
    res = {"workload": "cross_section", "data": "synthetic (device RAMBO)", "steps": args.steps,
           "warmup": args.warmup, "metric": METRIC, "unit": "points/s"}
    legs = [("k1_fp64", 1, "fp64", 1.0, 1 << 22), ("k4_mixed", 4, "mixed", 4.0, 1 << 22)]
    for name, k, prec, omega, n in legs:
        n = args.n_points or n
        plan = Plan(k, precision=prec)
        for _ in range(max(1, args.warmup)):
            cross_section(plan, omega, n, seed=77)
        t0 = time.perf_counter()
        for s in range(args.steps):
            r = cross_section(plan, omega, n, seed=78 + s)
        dt = (time.perf_counter() - t0) / args.steps
        leg = {"k": k, "precision": prec, "omega": omega, "n_points": n, "points_per_s": n / dt,
               "ms_per_step": dt * 1e3, "sigma": r["sigma"], "sigma_err": r["sigma_err"]}
        if k == 1:
            x = omega
            re2 = (1.0 / (4.0 * math.pi)) ** 2
            kn = 2.0 * math.pi * re2 * ((1 + x) / x ** 3 * (2 * x * (1 + x) / (1 + 2 * x) - math.log(1 + 2 * x))
                                        + math.log(1 + 2 * x) / (2 * x) - (1 + 3 * x) / (1 + 2 * x) ** 2)
            leg.update(klein_nishina=kn, pull=(r["sigma"] - kn) / r["sigma_err"])
        res[name] = leg
    res["value"] = res["k4_mixed"]["points_per_s"]
    res["config"] = {"workload": "cross_section", "k": "1 (FP64), 4 (mixed)", "n_points": "4,194,304 per step"}
    print(json.dumps(res), flush=True)


def run_abc(args):
    """The ABC model (paper App. F) through the same DAGs as QED with one spin
    state: points/s and FLOP rates of the node-reduced and the rewritten DAG,
    FP64 and mixed, for k = 1, 3, 5, 7, next to QED with one fixed state on
    the same k (the same DAG with 4x4 Dirac building blocks)."""
    import torch
    from paper_2511_19456_b300 import AbcPlan, Plan
    torch.cuda.set_device(0)
    res = {"workload": "abc", "data": "synthetic", "steps": args.steps, "warmup": args.warmup,
           "metric": METRIC, "unit": "points/s", "masses": ps.ABC_MASSES}
    fixed_hel = {1: [1, 2, -1, 1], 3: [1, 2, -1, 1, 2, 1], 5: [1, 2, -1] + [1, 2] * 2 + [1],
                 7: [1, 2, -1] + [1, 2] * 3 + [1]}
    for name, w in ps.ABC_WORKLOADS.items():
        k, n = w["k"], w["n_points"]
        mom = torch.from_numpy(ps.abc_workload_points(name)).cuda()
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        legs = {"n_points": n, "rs": w["rs"]}
        for dag in ("plain", "rewrite"):
            for prec in ("fp64", "mixed"):
                plan = AbcPlan(k, precision=prec, rewrite=dag == "rewrite", **ps.ABC_MASSES)
                ms = time_calls(lambda: plan.eval(mom, out), args.steps, args.warmup)
                fl = plan.info()["flops_per_point"]
                peak = PEAK_FP32_TFLOPS if prec == "mixed" else PEAK_FP64_TFLOPS
                legs[f"{dag}_{prec}"] = {"points_per_s": n / (ms * 1e-3), "ms": ms, "flops_per_point": fl,
                                         "tflops": fl * n / (ms * 1e-3) / 1e12,
                                         "frac_of_peak": fl * n / (ms * 1e-3) / 1e12 / peak}
        # QED, one fixed state, same k and DAG structure, QED kinematics
        qmom = torch.from_numpy(ps.points(k, n, 2.0 * k, w["seed"])).cuda()
        for prec in ("fp64", "mixed"):
            qp = Plan(k, summed=False, hel=fixed_hel[k], precision=prec)
            ms = time_calls(lambda: qp.eval(qmom, out), args.steps, args.warmup)
            legs[f"qed_fixed_plain_{prec}"] = {"points_per_s": n / (ms * 1e-3), "ms": ms,
                                               "flops_per_point": qp.info()["flops_per_point"]}
        legs["abc_over_qed_points_per_s_plain_fp64"] = (legs["plain_fp64"]["points_per_s"]
                                                       / legs["qed_fixed_plain_fp64"]["points_per_s"])
        res[name] = legs
    res["value"] = res["abc_k7"]["plain_fp64"]["points_per_s"]
    res["config"] = {"workload": "abc", "k": "1, 3, 5, 7", "dag": "plain and rewrite"}
    print(json.dumps(res), flush=True)


def run_sweep(args):
    """Node-reduction sweep (paper Sec. III-D, Fig. f_optimization): the CDAG
    of e- gamma -> e- + 4 gamma, one fixed spin state, FP64, executed node by
    node after 0, 10, ..., all 140 single node reductions.  For each state:
    nodes, FLOPs per point, points/s, the measured speed-up over the
    unreduced state and the one predicted from the FLOPs; then the scheduled
    kernel of the fully reduced DAG for comparison."""
    import torch
    from paper_2511_19456_b300 import Plan, TapePlan, reduction_steps
    torch.cuda.set_device(0)
    k = 4
    hel = [1, 2, -1] + [1 + (j % 2) for j in range(k)]
    n = args.n_points or 262144
    mom = torch.from_numpy(ps.points(k, n, 4.0, 2)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    S = reduction_steps(k)
    states = []
    for st in list(range(0, S, 10)) + [S]:
        plan = TapePlan(k, hel, st)
        inf = plan.info()
        ms = time_calls(lambda: plan.eval(mom, out), args.steps, args.warmup)
        states.append({"steps": st, "nodes": inf["nodes_reduced"], "compute_nodes": inf["compute_reduced"],
                       "flops_per_point": inf["flops_per_point"], "smem_bytes_per_team": inf["smem_bytes_per_team"],
                       "ms": ms, "points_per_s": n / (ms * 1e-3),
                       "tflops": inf["flops_per_point"] * n / (ms * 1e-3) / 1e12})
    for s_ in states:
        s_["speedup_measured"] = states[0]["ms"] / s_["ms"]
        s_["speedup_from_flops"] = states[0]["flops_per_point"] / s_["flops_per_point"]
    plan = Plan(k, summed=False, hel=hel)
    ms = time_calls(lambda: plan.eval(mom, out), args.steps, args.warmup)
    res = {"workload": "reduction_sweep", "data": "synthetic", "metric": METRIC, "unit": "points/s",
           "steps": args.steps, "warmup": args.warmup, "total_reductions": S, "states": states,
           "scheduled_reduced_kernel": {"points_per_s": n / (ms * 1e-3), "ms": ms,
                                        "speedup_over_unreduced_tape": states[0]["ms"] / ms},
           "value": states[-1]["points_per_s"],
           "config": {"workload": "reduction_sweep", "k": k, "n_points": n, "omega": 4.0, "hel": hel,
                      "precision": "fp64"}}
    print(json.dumps(res), flush=True)


def load_golden(name, per_point):
    """Rows of a stored oracle file under tests/golden (values the oracle
    wrote; reading them runs no oracle code)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return [rows[i:i + per_point] for i in range(0, len(rows), per_point)]


def config_legs(peaks, steps):
    """GPU legs of the four configurations other than the headline one,
    bounded to about a minute: throughput of both precisions (each plan
    tuned first), the fraction of the measured FMA peak, the adjoint where
    the configuration has one, and the GPU results on sample points.  Returns
    the records and the oracle checks that the cpu_baseline leg runs to fill
    in each error against the oracle."""
    import torch
    from paper_2511_19456_b300 import Batch, Plan, generate
    recs, checks = {}, []

    def peak(prec):
        return peaks["fp32_tflops"] if prec == "mixed" else peaks["fp64_tflops"]

    def leg(plan, n, ms, prec):
        tf = plan.info()["flops_per_point"] * n / (ms * 1e-3) / 1e12
        return {"n_points": n, "ms": ms, "points_per_s": n / (ms * 1e-3), "tflops": tf,
                "frac_of_measured_peak": tf / peak(prec)}

    # ---- k = 1, all 16 states, the 65,536 two-body points (FP64 config; mixed beside it)
    mom = ps.workload_points("compton_k1")
    d = torch.from_numpy(mom).cuda()
    out = torch.empty(len(mom), dtype=torch.float64, device="cuda")
    rec, got = {"config": "e- gamma -> e- gamma, 65,536 flat two-body points, omega = 1, all 16 states"}, {}
    for prec in ("mixed", "fp64"):
        plan = Plan(1, precision=prec)
        tuned = plan.tune(d)
        ms = time_calls(lambda: plan.eval(d, out), 4 * steps, 3)
        rec[prec] = dict(leg(plan, len(mom), ms, prec), kernel_form=tuned["form"], block=tuned["block"])
        got[prec] = out.cpu().numpy().copy()
    rec["speedup_mixed_vs_fp64"] = rec["fp64"]["ms"] / rec["mixed"]["ms"]
    recs["compton_k1"] = rec
    checks.append(("compton_k1", "error_vs_oracle", got, lambda o, m=mom: o.m2(m, kappa=True), "all 65,536 points"))

    # ---- k = 6, one fixed state, 262,144 points: forward and adjoint
    w = ps.WORKLOADS["compton_k6_fixed"]
    mom = ps.workload_points("compton_k6_fixed")
    d = torch.from_numpy(mom).cuda()
    out = torch.empty(len(mom), dtype=torch.float64, device="cuda")
    grad = torch.empty((len(mom), 6, 3), dtype=torch.float64, device="cuda")
    rec, got, gg = {"config": "e- gamma -> e- + 6 gamma, 262,144 RAMBO points, omega = 8, one fixed state "
                              f"{w['hel']}"}, {}, {}
    for prec in ("mixed", "fp64"):
        plan = Plan(6, summed=False, hel=w["hel"], precision=prec)
        st = steps if prec == "mixed" else 2
        ms = time_calls(lambda: plan.eval(d, out), st, 1)
        r = leg(plan, len(mom), ms, prec)
        got[prec] = out[:256].cpu().numpy().copy()
        ms_g = time_calls(lambda: plan.eval_grad(d, out, grad), st, 1)
        r.update(adjoint_ms=ms_g, adjoint_points_per_s=len(mom) / (ms_g * 1e-3), adjoint_over_forward_time=ms_g / ms)
        _, g32 = plan.eval_grad(d[:32].contiguous())
        gg[prec] = g32.cpu().numpy()
        rec[prec] = r
    rec["speedup_mixed_vs_fp64"] = rec["fp64"]["ms"] / rec["mixed"]["ms"]
    recs["compton_k6_fixed"] = rec
    hel = w["hel"]
    checks.append(("compton_k6_fixed", "error_vs_oracle", got,
                   lambda o, m=mom[:256]: o.m2(m, sum_mask=0, hel=hel, kappa=True), "the first 256 points"))
    checks.append(("compton_k6_fixed", "gradient_vs_oracle", gg,
                   lambda o, m=mom[:32]: o.grad(m, sum_mask=0, hel=hel), "the first 32 points"))

    # ---- the batched stream: 64 seeded requests, k = 1..5, one persistent launch (CUDA graph)
    reqs = ps.batched_requests()
    moms = [generate(r["k"], r["n_points"], r["omega"], r["seed"]) for r in reqs]
    n_tot = sum(r["n_points"] for r in reqs)
    rec = {"config": f"{len(reqs)} requests, k = 1..5, {n_tot} RAMBO points (generated on the device), "
                     "omega U[1, 8], all states"}
    host8 = [ps.points(r["k"], 8, r["omega"], r["seed"]) for r in reqs]
    got = {}
    for prec in ("mixed", "fp64"):
        plans = {k: Plan(k, precision=prec) for k in range(1, 6)}
        batch = Batch([plans[r["k"]] for r in reqs], [r["n_points"] for r in reqs])
        outs = batch.outputs()
        tuned_ms = batch.tune(moms, outs) if prec == "mixed" else None
        st, wu = (steps, 1) if prec == "mixed" else (1, 0)
        ms_b = time_calls(lambda: batch.eval(moms, outs), st, wu)
        seq_outs = [torch.empty_like(o) for o in outs]

        def seq():
            for r, m, o in zip(reqs, moms, seq_outs):
                plans[r["k"]].eval(m, o)
        ms_s = time_calls(seq, st, wu)
        flops = sum(plans[r["k"]].info()["flops_per_point"] * r["n_points"] for r in reqs)
        tf = flops / (ms_b * 1e-3) / 1e12
        rec[prec] = {"batched_ms": ms_b, "batched_points_per_s": n_tot / (ms_b * 1e-3), "tflops": tf,
                     "frac_of_measured_peak": tf / peak(prec), "sequential_ms": ms_s,
                     "sequential_points_per_s": n_tot / (ms_s * 1e-3), "launches_batched": 1,
                     "launches_sequential": len(reqs), "tune_best_ms": tuned_ms, "batch_info": batch.info()}
        # the first 8 points of every request, host-generated, through the same batched path
        small = Batch([plans[r["k"]] for r in reqs], [8] * len(reqs))
        so = small.eval([torch.from_numpy(h).cuda() for h in host8])
        got[prec] = np.concatenate([o.cpu().numpy() for o in so])
    rec["speedup_batched_mixed_vs_sequential_fp64"] = rec["fp64"]["sequential_ms"] / rec["mixed"]["batched_ms"]
    rec["speedup_batched_fp64_vs_sequential_fp64"] = rec["fp64"]["sequential_ms"] / rec["fp64"]["batched_ms"]
    recs["batched"] = rec

    def batched_oracle(o, hs=host8):
        parts = [o.m2(h, kappa=True) for h in hs]
        return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])
    checks.append(("batched", "error_vs_oracle", got, batched_oracle, "the first 8 points of each request"))

    # ---- k = 7, all 1024 states: forward and adjoint on slices, errors on the stored oracle points
    w = ps.WORKLOADS["compton_k7"]
    n_m, n_d = 16384, 2048
    mom = ps.points(7, n_m, w["omega"], w["seed"])
    d = torch.from_numpy(mom).cuda()
    out = torch.empty(n_m, dtype=torch.float64, device="cuda")
    grad = torch.empty((n_m, 7, 3), dtype=torch.float64, device="cuda")
    rec = {"config": f"e- gamma -> e- + 7 gamma, omega = 10, all 1024 states; timed on the first {n_m} (mixed) "
                     f"and {n_d} (FP64) of the workload's {w['n_points']} points; errors on 512 stored oracle points"}
    gold = load_golden("k7_summed_oracle.txt", 11)
    gmom = np.array([[[float(x) for x in row] for row in pt[1:]] for pt in gold]) if gold else None
    gold_g = load_golden("k7_summed_grad_oracle.txt", 8)
    for prec in ("mixed", "fp64"):
        plan = Plan(7, precision=prec)
        n = n_m if prec == "mixed" else n_d
        dd, oo, gr = d[:n], out[:n], grad[:n]
        ms = time_calls(lambda: plan.eval(dd, oo), 2 if prec == "mixed" else 1, 1)
        r = leg(plan, n, ms, prec)
        ms_g = time_calls(lambda: plan.eval_grad(dd, oo, gr), 2 if prec == "mixed" else 1, 1)
        r.update(adjoint_ms=ms_g, adjoint_points_per_s=n / (ms_g * 1e-3), adjoint_over_forward_time=ms_g / ms)
        if gold:
            ref = np.array([float(pt[0][0]) for pt in gold])
            kap = np.array([float(pt[0][1]) for pt in gold])
            m2 = plan.eval(torch.from_numpy(gmom).cuda()).cpu().numpy()
            r["error_vs_oracle"] = dict(error_stats(m2, ref, kap, prec), sample="512 stored oracle points")
        if gold_g:
            gref = np.array([[[float(x) for x in row] for row in pt[1:]] for pt in gold_g])
            _, g = plan.eval_grad(torch.from_numpy(np.ascontiguousarray(gmom[:len(gold_g)])).cuda())
            err = np.abs(g.cpu().numpy() - gref).max(axis=(1, 2)) / np.abs(gref).max(axis=(1, 2))
            r["gradient_vs_oracle"] = {"n": len(gold_g), "median": float(np.median(err)), "max": float(err.max()),
                                       "sample": "stored oracle dual-number gradients",
                                       "measure": "max |g - g_oracle| / max |g_oracle| per point"}
        rec[prec] = r
    rec["speedup_mixed_vs_fp64"] = (rec["mixed"]["points_per_s"] / rec["fp64"]["points_per_s"])
    recs["compton_k7"] = rec
    return recs, checks


def run_oracle_checks(recs, checks):
    """The oracle side of the configurations' error checks (part of the
    cpu_baseline leg: the oracle runs on the host cores only here)."""
    import oracle
    for cfg, key, got, fn, sample in checks:
        if key == "gradient_vs_oracle":
            _, gref = fn(oracle)
            res = {}
            for prec, g in got.items():
                err = np.abs(g - gref).max(axis=(1, 2)) / np.abs(gref).max(axis=(1, 2))
                res[prec] = {"n": int(err.size), "median": float(np.median(err)), "max": float(err.max()),
                             "measure": "max |g - g_oracle| / max |g_oracle| per point"}
        else:
            ref, kap = fn(oracle)
            res = {prec: error_stats(g, ref, kap, prec) for prec, g in got.items()}
        res["sample"] = sample
        recs[cfg][key] = res


def time_device(plan, d_mom, out, steps, warmup, stream, barrier, grad=None):
    """Device time per call of qed_eval (or, with a gradient buffer, of
    qed_eval_grad) with CUDA events on the launching stream."""
    import torch

    def call():
        if grad is None:
            plan.eval(d_mom, out, stream=stream)
        else:
            plan.eval_grad(d_mom, out, grad, stream=stream)
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / steps  # ms per step


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="compton_k4", choices=sorted(ps.WORKLOADS) + ["batched", "rewrite_vs_plain", "abc", "reduction_sweep", "cross_section"],
                    help="compton_k4 is the headline line; the others measure the other "
                         "configurations (adjoint at k = 6, k = 7, the batched stream)")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps of the FP64 path (default: --steps)")
    ap.add_argument("--fp64-points", type=int, default=None,
                    help="points of the FP64 legs of the non-headline workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle on the host cores (and with it every error against the oracle)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the other configurations (k = 1, k = 6 fixed, batched, k = 7)")
    ap.add_argument("--no-tune", action="store_true", help="time the plans' default kernel form and block")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only", choices=["mixed", "fp64"], default=None,
                    help="time one precision only (profiling runs)")
    ap.add_argument("--grad", action="store_true",
                    help="profiling runs (--only): time qed_eval_grad (|M|^2 and the adjoint) instead of qed_eval")
    ap.add_argument("--n-points", type=int, default=None,
                    help="override the workload's point count (profiling runs)")
    ap.add_argument("--dag", choices=["plain", "rewrite"], default="plain",
                    help="plain: the node-reduced DAG (one current per ordered photon prefix); "
                         "rewrite: the distributively rewritten DAG (one current per photon subset)")
    args = ap.parse_args()
    if args.impl == "reference":
        why = {"batched": "the batched stream is measured against the FP64 GPU path",
               "rewrite_vs_plain": "the rewritten DAG is measured against the plain DAG on the GPU",
               "abc": "the ABC model is measured against QED on the same DAGs on the GPU",
               "reduction_sweep": "the reduction sweep compares tapes on the GPU",
               "cross_section": "the cross section is checked against the closed-form Klein-Nishina value"}
        if args.workload in why:
            print(json.dumps({"impl": "reference", "unavailable": why[args.workload]}))
            return
        run_reference(args, args.workload)
        return
    if args.workload == "rewrite_vs_plain":
        run_rewrite_compare(args)
        return
    if args.workload == "abc":
        run_abc(args)
        return
    if args.workload == "reduction_sweep":
        run_sweep(args)
        return
    if args.workload == "cross_section":
        run_cross_section(args)
        return
    if args.workload != "compton_k4" and args.only is None and args.dag == "plain":
        run_other(args)
        return

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    barrier = (lambda: dist.barrier()) if ws > 1 else (lambda: None)

    from paper_2511_19456_b300 import Plan, measure_fma_peak
    from paper_2511_19456_b300.distributed import max_over_ranks

    w = ps.WORKLOADS[args.workload]
    k = w["k"]
    n = args.n_points or w["n_points"]
    mom = ps.points(k, n, w["omega"], w["seed"] + 7919 * rank)
    d_mom = torch.from_numpy(mom).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    hel = None if w["summed"] else w["hel"]

    res = {}
    launches = 0
    clocks = None
    fp64_steps = args.fp64_steps if args.fp64_steps is not None else args.steps
    legs = [("mixed", args.steps), ("fp64", fp64_steps)]
    if args.only:
        legs = [l for l in legs if l[0] == args.only]
    # the roofline denominators, measured on this GPU in this run
    peaks = measure_peaks(local) if not args.only else None
    for prec, steps in legs:
        plan = Plan(k, summed=w["summed"], hel=hel, precision=prec, rewrite=args.dag == "rewrite")
        # the autotuner (kernel form and block size), on a slice of the
        # workload, before the timed region
        tuned = plan.tune(d_mom[:min(n, 1 << 18)]) if not args.only and not args.no_tune else None
        info = plan.info()
        form = plan.kernel_form
        g_buf = torch.empty((n, k, 3), dtype=torch.float64, device="cuda") if args.grad and args.only else None
        with ClockSampler(local) as cs:
            ms = time_device(plan, d_mom, out, steps, args.warmup, stream, barrier, grad=g_buf)
        launches += steps
        ms = max_over_ranks(ms, device="cuda")
        pts = n * ws / (ms * 1e-3)
        flops = info["flops_per_point"]
        achieved = flops * n / (ms * 1e-3) / 1e12
        nominal = PEAK_FP32_TFLOPS if prec == "mixed" else PEAK_FP64_TFLOPS
        if peaks:
            peak = peaks["fp32_tflops"] if prec == "mixed" else peaks["fp64_tflops"]
            source = "measured: FMA chains on this GPU in this run (of measured)"
        else:
            peak, source = nominal, ("derived from unit counts and the 2032 MHz clock" if prec == "mixed"
                                     else "nominal B300 FP64 rate")
        res[prec] = {"value": pts, "ms_per_step": ms, "plan": plan, "info": info,
                     "out": out.cpu().numpy().copy() if not args.only else None,
                     "kernel": {"form": form, "block": info["block_threads"], "grid": info["grid_blocks"],
                                "tuned": tuned},
                     "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                                  "unit": "TFLOP/s", "frac": achieved / peak,
                                  "traffic": recorded_traffic(args.workload, prec, n, args.dag, form),
                                  "peak_source": source, "peak_nominal": nominal,
                                  "frac_of_nominal": achieved / nominal,
                                  "pipe": "FP32 FMA" if prec == "mixed" else "FP64 FMA",
                                  "flops_per_point": flops},
                     "clocks": cs.summary()}
        if prec == "mixed":
            clocks = cs.summary()

    if args.only:
        # profiling run: one precision, no end-to-end leg, a short line
        r = res[args.only]
        if rank == 0:
            print(json.dumps({"profile_run": args.only, "grad": args.grad, "workload": args.workload, "dag": args.dag,
                              "n_points": n, "kernel": r["kernel"],
                              "ms_per_step": r["ms_per_step"], "value": r["value"],
                              "roofline": r["roofline"]}), flush=True)
        if ws > 1:
            dist.destroy_process_group()
        return

    # end to end through the public API on pinned host buffers
    e2e = None
    if not args.no_e2e:
        plan = res["mixed"]["plan"]
        h_mom = torch.from_numpy(mom).pin_memory()
        h_out = torch.empty(n, dtype=torch.float64).pin_memory()
        for _ in range(max(1, args.warmup)):
            plan.eval_host(h_mom, h_out)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            plan.eval_host(h_mom, h_out)
        e2e_s = (time.perf_counter() - t0) / args.steps
        launches += args.steps * len(host_chunks(n))
        e2e_s = max_over_ranks(e2e_s, device="cuda")
        e2e = {"value": n * ws / e2e_s, "unit": "points/s",
               "h2d_bytes_per_step": int(h_mom.numel() * 8),
               "d2h_bytes_per_step": int(h_out.numel() * 8)}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return
    mixed, fp64 = res["mixed"], res["fp64"]
    line = {
        "metric": METRIC,
        "value": mixed["value"],
        "unit": "points/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": mixed["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "dag": args.dag, "k": k, "n_points": n, "omega": w["omega"],
                   "states_summed": mixed["info"]["n_states"], "diagrams": mixed["info"]["n_diagrams"],
                   "generator": "RAMBO (seeded SplitMix64)" if k > 1 else "flat 2-body",
                   "l2": f"inputs {n * (k + 3) * 32 / 1e6:.0f} MB per step, larger than the 126 MB L2",
                   "precision": "mixed: FP32 currents and Kahan diagram sums; FP64 momenta, "
                                "denominators, spin sum"},
        "kernel": mixed["kernel"],
        "roofline": mixed["roofline"],
        "fp64": {"value": fp64["value"], "unit": "points/s", "ms_per_step": fp64["ms_per_step"],
                 "steps": fp64_steps, "kernel": fp64["kernel"], "roofline": fp64["roofline"],
                 "clocks": fp64["clocks"]},
        "speedup_mixed_vs_fp64": mixed["value"] / fp64["value"],
        "peaks_measured": peaks,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    # the adjoint (qed_eval_grad) of the same plans, on slices of the workload
    if not args.no_configs:
        adj = {"sample": "the first 262,144 (mixed) and 65,536 (FP64) points of the workload"}
        for prec, nn in (("mixed", min(n, 1 << 18)), ("fp64", min(n, 1 << 16))):
            plan = res[prec]["plan"]
            mm = d_mom[:nn]
            oo = torch.empty(nn, dtype=torch.float64, device="cuda")
            gg = torch.empty((nn, k, 3), dtype=torch.float64, device="cuda")
            ms_f = time_calls(lambda: plan.eval(mm, oo), 3, 1)
            ms_g = time_calls(lambda: plan.eval_grad(mm, oo, gg), 3, 1)
            adj[prec] = {"n_points": nn, "points_per_s": nn / (ms_g * 1e-3), "ms": ms_g,
                         "forward_ms": ms_f, "adjoint_over_forward_time": ms_g / ms_f}
        line["adjoint"] = adj
    checks = []
    if not args.no_configs:
        line["configs"], checks = config_legs(peaks, steps=3)
    if not args.no_cpu_baseline:
        line["cpu_baseline"], sample = cpu_baseline(mom, k)
        if sample is not None:
            idx, ref, kap = sample
            line["error_vs_oracle"] = {
                "sample": f"the cpu_baseline leg's {len(idx)} points (workload points {idx[0]}..{idx[-1]})",
                "mixed": error_stats(mixed["out"][idx], ref, kap, "mixed"),
                "fp64": error_stats(fp64["out"][idx], ref, kap, "fp64")}
        run_oracle_checks(line.get("configs", {}), checks)
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
