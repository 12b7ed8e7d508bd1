#!/usr/bin/env python3
"""Throughput of binned photon-number distributions on the GPU.

Metric: generating-function points per second (every point of the roots-of-unity grid
counts; conjugate symmetry means about half are evaluated) and binned P(b) tables per
second, for the FP32-arithmetic path (``value``) next to the FP64 path (``fp64``), both held
to |P - P_oracle| <= 1e-10 and both as a user gets them (automatic kernel choice).

Workload (the largest single-problem configuration): M = 24 spatial x K = 4 internal
(Schmidt) modes per source with weights lambda_k ~ exp(-k/2), each source in its own seeded
Haar internal basis (so the 192 x 192 matrices are dense), T = sqrt(0.6) U with U Haar,
displacement alpha ~ CN(0, 0.1) on 4 inputs, 3 detector groups of 8, N_l = 20: 21^3 = 9261
grid points of 192 x 192 complex matrices per table.  One step = one table: every device
stage of the path (grid phases, the factorisations - shared block eliminations down the
tree of the grid's axes, or one LU per point - the log det / exponent epilogue, the inverse
DFT, the diagnostics) with the state resident in HBM.  ``e2e`` times the public C ABI from
host buffers: per step the host FP64 state algebra and upload (gbsbin_plan_set_state), the
execute and the copy of the table back.  The n = 32 grid (four groups), the 256-problem
batch, the n = 200 gradient, the M = 256 total photon number, Fock inputs and App. D are
timed as extras.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD_INDEX = 2
WORKLOAD_NAME = "M24_K4_L3_N20_n192_9261pts"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
SMS = 152
SM_MAX_MHZ = 2070.0
FP32_LANES_PER_SM = 128
FP64_FMA_PER_SM_CLK = 2      # 1.25 TFLOP/s nominal / (152 SMs x 2.07 GHz x 2 flops)
METRIC = "generating-function points/s (binned P(b) tables/s alongside), FP32+refine vs FP64"


def algorithmic_flops(n: int, has_gamma: bool) -> float:
    """Per evaluated point, the work the method needs whatever the precision: the complex
    unpivoted LU, (8/3) n^3 real flops, plus 8 n^2 for the two triangular solves of the
    exponent when the state is displaced."""
    n = float(n)
    return (8.0 / 3.0) * n ** 3 + (8.0 * n * n if has_gamma else 0.0)


def tree_work(prob, n_eval: int, has_gamma: bool):
    """The tree of block eliminations (kernels 11 and 12): complex multiply-adds per table.  Level l
    (one node per combination of the first l axes' roots) runs a Gauss-Jordan sweep over nb
    pivot columns of its m x (m + 1) augmented matrix: step kk scales row kk right of the
    pivot and updates the other m - 1 rows there, (m - kk)(m + 1 - kk - 1) multiply-adds,
    plus the fill (nb (m + 1) products) and the u update (nb (m - nb)); each leaf runs an
    unpivoted LU of its NL x NL block with the right-hand side, sum (NL - kk)^2, and, if
    displaced, the back substitution (NL^2 / 2).  Returns (complex MACs, level launches)."""
    rows = [2 * prob.K * int(np.sum(prob.bin_of_mode == l)) for l in range(prob.L)]
    m, nodes, macs = prob.n, 1, 0.0
    for l in range(prob.L - 1):
        nodes *= int(prob.radix[l])
        nb, cols = rows[l], m + 1
        per = nb * cols + sum((m - kk) * (cols - kk - 1) for kk in range(nb))
        if has_gamma:
            per += nb * (m - nb)
        macs += nodes * per
        m -= nb
    per_leaf = sum((m - kk) ** 2 for kk in range(m)) + (m * m / 2.0 if has_gamma else 0.0)
    macs += n_eval * per_leaf
    return macs, tree_level_launches(prob.radix, prob.L)


def btree_work(prob, n_eval: int, has_gamma: bool, smem_slots: int = 200 * 1024 // 16):
    """The large-matrix tree (kernels 13 and 14): complex multiply-adds per table, as the library
    counts them.  Conjugate symmetry halves either the last axis (the leaves) or the first
    (then every level's nodes halve and each leaf covers a point or its conjugate); the
    library takes the halving with fewer multiply-adds.  Level l eliminates its group's nb
    pivots in sub-steps of nbs (as many as fit the shared-memory budget: nbs (D + 1) <= 12800
    16-byte slots, D the augmented dimension): the pivot rows among themselves,
    sum (nbs - kk - 1)(D - kk - 1), and each of the other D - nbs rows against them,
    sum (D - kk - 1); per leaf parent a Householder reduction to Hessenberg form, sum over k of
    2 (m - k - 1)(m - k + 1) + 2 m (m - k - 1); per leaf the Hessenberg elimination, m^2 / 2
    (twice that when displaced)."""
    rows = [2 * prob.K * int(np.sum(prob.bin_of_mode == l)) for l in range(prob.L)]
    radix = [int(r) for r in prob.radix]
    best = None
    for halve_first in (0, 1):
        cnt = list(radix)
        if halve_first:
            cnt[0] = radix[0] // 2 + 1
        else:
            cnt[-1] = radix[-1] // 2 + 1
        m, nodes, macs = prob.n, 1, 0.0
        for l in range(prob.L - 1):
            nodes *= cnt[l]
            D = m + 1
            cap = min(128, smem_slots // (D + 1))
            nsub = -(-rows[l] // cap)
            per = -(-rows[l] // nsub)
            p0 = 0
            while p0 < rows[l]:
                nbs = min(per, rows[l] - p0)
                top = sum((nbs - kk - 1) * (D - kk - 1) for kk in range(nbs))
                row = sum(D - kk - 1 for kk in range(nbs))
                macs += nodes * (top + (D - nbs) * row)
                D -= nbs
                p0 += nbs
            m -= rows[l]
        hess = sum(2.0 * (m - k - 1) * (m - k + 1) + 2.0 * m * (m - k - 1) for k in range(m - 2))
        macs += nodes * hess
        macs += nodes * cnt[-1] * (2.0 if has_gamma else 1.0) * m * m / 2.0
        best = macs if best is None else min(best, macs)
    return best


def tree_level_launches(radix, L, num_sms=SMS, span_max=4):
    """Level launches of the tree: a level whose children would fill fewer than half the SMs
    takes the next level into the same launch (up to span_max groups, while a level remains
    before the leaves), as the library's launch sequence does."""
    launches, nodes, l = 0, 1, 0
    while l + 1 < L:
        children, span = nodes * int(radix[l]), 1
        while span < span_max and l + span + 1 < L and 2 * children < num_sms:
            children *= int(radix[l + span])
            span += 1
        launches += 1
        nodes = children
        l += span
    return launches


def pipe_flops(n: int, has_gamma: bool, precision: int) -> float:
    """Per evaluated point, the arithmetic-pipe work the kernel issues, in FP32-FMA
    equivalents x 2 (so that it compares with a flop peak).  FP64: as algorithmic_flops.
    FP32R: LU 4 FMA per complex MAC over n^3/3 MACs; exact residual 3 mad.wide.s32 per
    complex MAC over n^3/3 MACs, each worth 2 FMA slots (it issues at half the FP32 FMA
    rate), plus ~30 integer operations per entry; Z = L^^-1 E (n^3/2 complex MACs) and
    diag(U^^-1 Z) (n^3/6) at 4 FMA per MAC; if displaced, four triangular solves (8 n^2)
    and the solve residual by Dot2 (80 n^2)."""
    n = float(n)
    if precision == 0:
        return algorithmic_flops(n, has_gamma)
    slots = (4.0 / 3.0 + 2.0 + 2.0 + 2.0 / 3.0) * n ** 3 + 30.0 * n * n
    if has_gamma:
        slots += 8.0 * n * n + 80.0 * n * n
    return 2.0 * slots


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max([num(r[3]) for r in rows if num(r[3]) is not None], default=None)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args):
    """CPU oracle as the reference arm: same workload and metric, each step a bounded
    sample of grid points evaluated by the oracle on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    prob = synth.config(WORKLOAD_INDEX)
    XA, gamma, labels = oracle.plan(prob)
    radix = prob.radix
    npts = prob.n_points
    rng = np.random.default_rng(0)
    all_digits = np.stack(np.unravel_index(np.arange(npts), tuple(radix)), axis=1)
    # size the sample so the whole run stays within about two minutes
    t0 = time.perf_counter()
    oracle.logq_points(XA, gamma, labels, radix, all_digits[:512])
    per_point = (time.perf_counter() - t0) / 512
    budget = 120.0 / max(1, args.steps + args.warmup)
    sample = int(max(64, min(npts, budget / per_point)))
    for _ in range(args.warmup):
        oracle.logq_points(XA, gamma, labels, radix, all_digits[rng.choice(npts, sample, replace=False)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.logq_points(XA, gamma, labels, radix, all_digits[rng.choice(npts, sample, replace=False)])
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "n": prob.n, "grid_points": npts},
            "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} random grid points of the {npts}-point grid per step"},
            "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_plan(gb, torch, plan, table, stream, flush, steps, world):
    """CUDA events around `steps` executes of one plan on `stream` (L2 flushed between steps,
    outside the events), with the library's own point-kernel events read back after each
    step; max over ranks."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kms = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    st, d = 0, None
    for s in range(steps):
        flush.zero_()
        ev[s][0].record(stream)
        gb.gbsbin_execute(plan.handle, table, stream)
        ev[s][1].record(stream)
        st, d = gb.gbsbin_diagnostics(plan.handle, stream)   # syncs; reads the kernel time
        kms.append(d["point_kernel_ms"])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    gpu_ms = sum(a.elapsed_time(b) for a, b in ev)
    if world > 1:
        t = torch.tensor([gpu_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        gpu_ms = float(t.item())
    return {"gpu_ms": gpu_ms, "ms_per_step": gpu_ms / steps, "kernel_ms": float(np.mean(kms)), "status": st,
            "diag": d, "wall_s": t_wall, "steps": steps}


def _side_steps(gb, torch, plan, table, stream, steps, budget_s=8.0):
    """Steps for a plan timed beside the headline: as many as fit in ~budget_s, at most
    `steps`, at least 3."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gb.gbsbin_execute(plan.handle, table, stream)
    torch.cuda.synchronize()
    one = max(time.perf_counter() - t0, 1e-6)
    return int(max(3, min(steps, budget_s / one)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (n=32 grid, 256-problem batch, n=200 gradient, "
                         "M=256 total photon number, Fock inputs, App. D fine-grained)")
    ap.add_argument("--extras", default="n32,batch,n200,e3,fock,herald,moments,appd",
                    help="comma list of the other workloads to time: n32, batch, n200, e3, fock, herald, moments, appd")
    ap.add_argument("--extra-steps", type=int, default=3)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2412_17742_gb300 as gb
    if rank == 0:
        from paper_2412_17742_gb300 import build as libbuild
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    gb.load()

    prob = synth.config(WORKLOAD_INDEX)
    npts = prob.n_points
    n = prob.n
    has_gamma = prob.alpha is not None
    stream = torch.cuda.current_stream()
    # precision 1 (FP32 arithmetic) and precision 0 (FP64) as a user gets them (automatic
    # kernel choice), and the per-point blocked FP32 + refinement kernel beside them
    plans = {1: gb.Plan(prob, precision=1, want_timing=True), 0: gb.Plan(prob, precision=0, want_timing=True)}
    if plans[1].diagnostics(stream)[1]["kernel_name"] != "blk_fp32r":
        plans["blk"] = gb.Plan(prob, precision=1, want_timing=True, tile_override=6)
    tables = {p: torch.empty(plans[p].shape, dtype=torch.float64, device="cuda") for p in plans}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    peaks_meas = {"fp64_tflops": gb.gbsbin_alu_peak(0, SMS * 8), "fp32_tflops": gb.gbsbin_alu_peak(1, SMS * 8),
                  "int64_mad_wide_tops": gb.gbsbin_alu_peak(2, SMS * 8)}

    for p in plans:
        for _ in range(max(args.warmup, 3)):
            gb.gbsbin_execute(plans[p].handle, tables[p], stream)
    torch.cuda.synchronize()
    steps = {p: (args.steps if p == 1 else _side_steps(gb, torch, plans[p], tables[p], stream, args.steps))
             for p in plans}

    sampler = ClockSampler(local)
    sampler.start()
    results = {p: _time_plan(gb, torch, plans[p], tables[p], stream, flush, steps[p], world) for p in plans}
    clocks = sampler.stop()

    # end to end through the C ABI with host buffers: per step the host FP64 state algebra
    # and upload (gbsbin_plan_set_state), the execute and the copy of the table back
    host_outs = [torch.empty(plans[1].shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    args_prob = gb.ProblemArgs(prob)
    d1 = results[1]["diag"]
    h2d = d1["state_upload_bytes"]
    d2h = int(np.prod(plans[1].shape)) * 8
    for _ in range(3):
        gb.gbsbin_plan_set_state(plans[1].handle, args_prob, stream)
        gb.gbsbin_execute_host(plans[1].handle, host_outs[0], stream)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.e2e_steps, int(10.0 / max(results[1]["ms_per_step"] * 1e-3, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):                        # each call returns with the table on the host
        gb.gbsbin_plan_set_state(plans[1].handle, args_prob, stream)
        gb.gbsbin_execute_host(plans[1].handle, host_outs[0], stream)
    torch.cuda.synchronize()
    e2e_sync_value = world * npts * e2e_steps / (time.perf_counter() - t0)
    # pipelined: the host algebra and upload of step i + 1 overlap the device work of step i
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        gb.gbsbin_plan_set_state(plans[1].handle, args_prob, stream)
        gb.gbsbin_execute_host_async(plans[1].handle, host_outs[i & 1], stream)
    torch.cuda.synchronize()
    e2e_value = world * npts * e2e_steps / (time.perf_counter() - t0)

    out_points = {p: world * npts * results[p]["steps"] / (results[p]["gpu_ms"] * 1e-3) for p in results}
    flops_pt = algorithmic_flops(n, has_gamma)
    peak32 = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    peak64 = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    tf32_peak = _measured_peaks().get("bf16_tflops", 1973.9) / 2.0   # dense TF32 = BF16 / 2 (nominal ratio)

    def roofline(p, peak, peak_source):
        r, d = results[p], results[p]["diag"]
        achieved = flops_pt * d["n_evaluated"] / (r["kernel_ms"] * 1e-3) / 1e12
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "traffic": _profiled_traffic(d["kernel_name"]), "kernel": d["kernel_name"],
               "kernel_ms": r["kernel_ms"], "peak_source": peak_source,
               "flops": "method's per-point work: complex unpivoted LU (8/3) n^3 + 8 n^2 exponent solves, "
                        "per evaluated point", "flops_per_point": flops_pt, "units_per_launch": d["n_evaluated"]}
        issued = _issued_work(prob, d, p != 0 and d["kernel_name"] != "gmem_fp64")
        if issued:
            name, ops, unit, pk = issued
            out.update({"issued": name, "issued_rate": ops / (r["kernel_ms"] * 1e-3) / 1e12,
                        "issued_unit": unit, "issued_peak": pk,
                        "issued_frac": ops / (r["kernel_ms"] * 1e-3) / 1e12 / pk})
        stale = _traffic_note(d["kernel_name"])
        if stale:
            out["traffic_note"] = stale
        return out

    line = {
        "metric": METRIC, "value": out_points[1], "unit": "points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": results[1]["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2" if d1["kernel_name"].endswith("df32") else "f32+f64refine", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "n": n, "grid_points": npts, "evaluated_points": d1["n_evaluated"],
                   "bins": prob.L, "cutoff": int(prob.cutoff[0]), "internal_modes": prob.K, "displaced": has_gamma,
                   "precision": "fp32_refine", "kernel": d1["kernel_name"],
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas{world}"},
        "tables_per_s": world * results[1]["steps"] / (results[1]["gpu_ms"] * 1e-3),
        "fp64": {"value": out_points[0], "unit": "points/s", "ms_per_step": results[0]["ms_per_step"],
                 "steps": results[0]["steps"],
                 "tables_per_s": world * results[0]["steps"] / (results[0]["gpu_ms"] * 1e-3),
                 "point_kernel_ms": results[0]["kernel_ms"], "kernel": results[0]["diag"]["kernel_name"],
                 "roofline": roofline(0, peak64, "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2070 MHz")},
        "speedup_fp32r_vs_fp64": out_points[1] / out_points[0],
        "roofline": dict(roofline(1, peak32, "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"),
                         tensor_peak=tf32_peak, tensor_frac=None,
                         tensor_note="TF32 dense peak (measured BF16 burst / 2) for context; the point stage "
                                     "issues no tensor-core instructions on this path",
                         measured_alu_chains=peaks_meas),
        "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps,
                "mode": "pipelined: set_state + execute_host_async per step, one synchronise at the end"},
        "e2e_sync": {"value": e2e_sync_value, "unit": "points/s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h, "mode": "set_state + execute_host (synchronous) per step"},
        "gpu_launches": int(d1["launches"]) * args.steps,
        "clocks": clocks,
        "diagnostics": {"sum_P": d1["sum_P"], "min_pivot_re": d1["min_pivot_re"],
                        "bad_points": d1["n_bad_points"], "fp64_sum_P": results[0]["diag"]["sum_P"]},
    }
    if "blk" in results:
        rb = results["blk"]
        line["per_point_fp32_refine"] = {"kernel": rb["diag"]["kernel_name"], "value": out_points["blk"],
                                         "unit": "points/s", "ms_per_step": rb["ms_per_step"],
                                         "steps": rb["steps"], "point_kernel_ms": rb["kernel_ms"],
                                         "roofline": roofline("blk", peak32, "derived FP32 peak")}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"], errs = cpu_baseline(prob, args.cpu_seconds, tables)
        line["max_abs_err_vs_oracle"] = errs
    for p in plans.values():
        p.close()
    if not args.no_extras:
        which = {w.strip() for w in args.extras.split(",") if w.strip()}
        line["workloads"] = extra_workloads(gb, torch, stream, flush, args.extra_steps, world, which)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def _issued_work(prob, d, fp32):
    """The arithmetic-pipe work the kernel issues per launch, where it differs from the
    method's flops: (description, operations, unit, peak).  Per-point FP32 + refinement
    kernels: pipe_flops against the FP32 peak.  Trees: complex multiply-adds x 64 FP32-pipe
    operations (pairs) against the FP32 issue rate, or x 8 flops (FP64) against the FP64 peak."""
    name = d["kernel_name"]
    n = prob.n
    has_gamma = prob.alpha is not None
    issue32 = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak32 = 2 * issue32
    peak64 = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    if name in ("tree_df32", "tree_fp64"):
        macs, _ = tree_work(prob, d["n_evaluated"], has_gamma)
        if name == "tree_df32":
            return ("tree complex multiply-adds x 64 FP32-pipe operations", 64.0 * macs, "T ops/s", issue32)
        return ("tree complex multiply-adds x 8 FP64 flops", 8.0 * macs, "TFLOP/s", peak64)
    if name in ("btree_df32", "btree_fp64"):
        macs = btree_work(prob, d["n_evaluated"], has_gamma)
        if name == "btree_df32":
            return ("tree complex multiply-adds x 64 FP32-pipe operations", 64.0 * macs, "T ops/s", issue32)
        return ("tree complex multiply-adds x 8 FP64 flops", 8.0 * macs, "TFLOP/s", peak64)
    if fp32 and name.endswith("fp32r"):
        return ("FP32-FMA-slot equivalents x 2 of the LU, exact residual and trace correction",
                pipe_flops(n, has_gamma, 1) * d["n_evaluated"], "TFLOP/s", peak32)
    return None


def _traffic_note(kernel_name):
    """Why `traffic` is null, said out loud: no capture of this kernel, or its sources
    changed since the committed capture (the figure of that capture is quoted)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        entry = json.load(open(path)).get(kernel_name)
    except (OSError, ValueError):
        return "no profiles/traffic.json"
    if not entry:
        return f"no DRAM capture of {kernel_name} in profiles/traffic.json"
    try:
        if _sources_hash(entry["sources"]) != entry["sources_hash"]:
            return (f"stale: sources changed since the capture (captured "
                    f"{entry.get('dram_bytes_per_launch', entry.get('dram_bytes_per_table'))} B per launch)")
    except (OSError, KeyError):
        return "capture record unreadable"
    return None


def _timed(torch, stream, flush, steps, fn):
    """Sum of CUDA-event durations of `steps` calls of fn on `stream`, L2 flushed between."""
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    return total


def extra_workloads(gb, torch, stream, flush, steps, world, which=("n32", "batch", "n200", "e3")):
    """The other workloads, a few steps each: per-table and per-point rates, FP32R next to
    FP64 where both apply."""
    out = {}
    if "n32" in which:
        out.update(_extra_n32(gb, torch, stream, flush, max(steps, 200), world))
    if "batch" in which:
        out.update(_extra_batch(gb, torch, stream, flush, steps, world))
    if "n200" in which:
        out.update(_extra_n200(gb, torch, stream, flush, steps, world))
    if "e3" in which:
        out.update(_extra_e3(gb, torch, stream, flush, steps, world))
    if "fock" in which:
        out.update(_extra_fock(gb, torch, stream, flush, steps, world))
    if "herald" in which:
        out.update(_extra_herald(gb, torch, stream, flush, steps, world))
    if "moments" in which:
        out.update(_extra_moments(gb, torch, steps))
    if "appd" in which:
        try:
            out.update(_extra_distinguishable(gb, torch, steps))
        except Exception as ex:                           # reported, never fatal to the bench line
            out["appd_distinguishable_m16_ones"] = {"error": str(ex)[:200]}
    return out


def _extra_herald(gb, torch, stream, flush, steps, world):
    """Heralded states (Sec. VII): the Fock-state source of Sec. VIII (two ports x two spectral
    modes, spectral purity 0.9, no loss; one port heralds with its spectral modes summed, cutoff
    3, the kept mode to Fock cutoff 15, 16-fold oversampled grid of 64 points) and a larger one
    (16 ports x 2 internal modes, two heralding groups of six ports, cutoff 8 each: 81 points;
    two kept modes to Fock cutoff 6: 2401 coefficients per point), per execute (the point
    kernel and the inverse DFT over the heralding axes), CUDA events, L2 flushed; and the
    fidelity of the heralded single photon from the GPU's own state."""
    out = {}
    cases = [("fock_source_p0.9", synth.fock_heralding_source(0.9, 1.0), synth.FOCK_HERALD_ROLES, [3], 15, 16)]
    prob, roles, cut, fc = synth.herald_config()
    cases.append(("m16_k2_two_groups_two_kept", prob, roles, cut, fc, 1))
    for name, prob, roles, cut, fc, over in cases:
        with gb.HeraldPlan(prob, roles, cut, fc, oversample=over) as h:
            rho = torch.empty(h.shape, dtype=torch.complex128, device="cuda")
            pr = torch.empty(h.prob_shape, dtype=torch.float64, device="cuda")
            run = lambda: gb.gbsbin_herald_execute(h.handle, rho, pr, stream)
            for _ in range(3):
                run()
            k = max(steps, 20)
            ms = _timed(torch, stream, flush, k, run) / k
            d = h.diagnostics(stream)
            entry = {"ms_per_execute": ms, "grid_points": d["n_points"], "rho_elements": d["table_size"],
                     "points_per_s": world * d["n_points"] / (ms * 1e-3), "launches": d["launches"],
                     "sum_Pr": d["sum_P"], "status": d["status"]}
            if name.startswith("fock"):
                r, p = rho.cpu().numpy(), pr.cpu().numpy()
                entry["fidelity_n1"] = float(np.sqrt((r[1, 1, 1] / p[1]).real))
            out[name] = entry
    return {"herald": out}


def _extra_moments(gb, torch, steps):
    """Cumulant tensors of orders 1-4 of the binned counts on the GPU (FP64) for the n = 192
    workload (three groups) and n = 512 (M = 256, eight groups): the device time of the launches
    (CUDA events inside the call), the whole call (host state algebra, uploads, allocation), the
    host evaluators' time for the same four tensors, and the largest relative difference.
    Roofline on the complex multiply-adds: n^2 (n + 32) / 2 for the Hermitian Y_b (the tiles on
    and above the diagonal) and L^2 n^2 / 2 for the C_4 traces, x 8 FP64 flops, against the
    derived FP64 peak."""
    out = {}
    rng = np.random.default_rng(77)
    cases = [("n192_L3", synth.config(2)),
             ("n512_L8", synth.random_problem(rng, 256, 1, 8, 2, displaced=True, r_range=(0.3, 0.9)))]
    peak64 = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    for name, prob in cases:
        gb.gbsbin_cumulants_device(prob)                       # warm-up
        k = max(3, min(steps, 10))
        dev_ms, t0 = [], time.perf_counter()
        for _ in range(k):
            outs, ms = gb.gbsbin_cumulants_device(prob, with_time=True)
            dev_ms.append(ms)
        call_ms = (time.perf_counter() - t0) / k * 1e3
        entry = {"n": 2 * prob.M * prob.K, "groups": int(prob.L), "device_ms": float(np.median(dev_ms)),
                 "call_ms": call_ms, "precision": "fp64"}
        gb.gbsbin_cumulants_device(prob, precision=gb.GBSBIN_FP32_REFINE)
        pair_ms = [gb.gbsbin_cumulants_device(prob, precision=gb.GBSBIN_FP32_REFINE, with_time=True)[1]
                   for _ in range(k)]
        pairs = gb.gbsbin_cumulants_device(prob, precision=gb.GBSBIN_FP32_REFINE)
        entry["fp32_pairs"] = {"device_ms": float(np.median(pair_ms)),
                               "max_rel_diff_vs_fp64": max(float(np.abs(a - b).max() / np.abs(b).max())
                                                           for a, b in zip(pairs, outs))}
        n, L = entry["n"], entry["groups"]
        flops = 8.0 * (n * n * (n + 32) / 2.0 + L * L * n * n / 2.0)
        entry["roofline"] = {"bound": "alu", "achieved": flops / (entry["device_ms"] * 1e-3) / 1e12, "peak": peak64,
                             "unit": "TFLOP/s", "peak_source": "derived FP64 peak"}
        entry["roofline"]["frac"] = entry["roofline"]["achieved"] / peak64
        if n <= 192:
            t0 = time.perf_counter()
            mean, cov = gb.gbsbin_moments(prob)
            host = [mean, cov, gb.gbsbin_cumulants3(prob), gb.gbsbin_cumulants4(prob)]
            entry["host_ms"] = (time.perf_counter() - t0) * 1e3
            entry["max_rel_diff_vs_host"] = max(float(np.abs(a - b).max() / np.abs(b).max()) for a, b in zip(outs, host))
        out[name] = entry
    return {"cumulants_device": out}


def _extra_distinguishable(gb, torch, steps):
    """App. D's fine-grained Pr(n) of a fully distinguishable state (16 sources, each in its own
    internal mode, r ~ U(0.5, 0.9), lossy Haar interferometer; one photon per detector: 2^16 =
    65536 evaluation points, N = 16): the device sum (one thread per point, FP64, compensated)
    against the host sum in Gray-code order, per call (the device call includes its buffer
    allocation); both values with their rounding-error estimates."""
    rng = np.random.default_rng(1700)
    M = 16
    r = np.diag(rng.uniform(0.5, 0.9, M))
    T = np.sqrt(rng.uniform(0.4, 0.9, M))[:, None] * synth.haar_unitary(M, rng)
    prob = synth.Problem(M, M, r, T, np.arange(M, dtype=np.int32), np.full(M, 1, np.int32))
    pattern = [1] * M
    gb.gbsbin_prob_distinguishable_device(prob, pattern)       # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        dev, dev_err = gb.gbsbin_prob_distinguishable_device(prob, pattern, with_error=True)
    t_dev = (time.perf_counter() - t0) / steps
    t0 = time.perf_counter()
    host, host_err = gb.gbsbin_prob_distinguishable(prob, pattern, with_error=True)
    t_host = time.perf_counter() - t0
    pts = 2 ** M
    return {"appd_distinguishable_m16_ones": {"points": pts, "N": M, "device_ms_per_call": t_dev * 1e3,
                                           "device_points_per_s": pts / t_dev, "host_ms": t_host * 1e3,
                                           "host_points_per_s": pts / t_host, "prob_device": dev,
                                           "prob_device_abs_err_estimate": dev_err, "prob_host": host,
                                           "prob_host_abs_err_estimate": host_err, "precision": "fp64"}}


def _extra_fock(gb, torch, stream, flush, steps, world):
    """Fock inputs through a lossy circuit (App. C): 16 single photons in 32 ports, output
    loss eta_i ~ U(0.4, 0.9), three detector groups, the whole table (N_l = 16): 2^15 input
    nodes x 2601 output-group points.  FP64 kernel against FP32 pairs; the pipe operations
    per (node, point) pair are counted from the kernels' inner loop (FP64: 2L additions and
    4 multiply-adds per photon plus 2; FP32 pairs: 4L additions, 12 for the renormalisation
    and 38 per product per photon, plus 16)."""
    fp = synth.fock_config()
    nin = int(np.count_nonzero(fp.photons))
    L = fp.L
    nodes = 1
    for c in sorted(fp.photons[fp.photons > 0])[1:]:
        nodes *= int(c) + 1
    radix = [int(c) + 1 for c in fp.cutoff]
    half = radix[-1] // 2 + 1
    points = int(np.prod(radix[:-1])) * half
    pairs = nodes * points
    N = int(fp.photons.sum())
    ops = {"fp64": nin * 2 * L + 4 * N + 2, "df32": nin * (4 * L + 12) + 38 * N + 16}
    peaks = {"fp64": (0.5 * 1.05e12, "FP64 pipe: measured 1.05 TFLOP/s dependent-FMA rate / 2"),
             "df32": (152 * 128 * 2.07e9, "FP32 pipe: 152 SMs x 128 lanes x 2070 MHz")}
    res = {"nodes": nodes, "points": points, "occupied_inputs": nin}
    tables = {}
    for name, prec in (("fp64", 0), ("df32", 1)):
        with gb.FockPlan(fp, precision=prec, want_timing=True) as p:
            t = torch.empty(p.shape, dtype=torch.float64, device="cuda")
            gb.gbsbin_fock_execute(p.handle, t, stream)
            ms = _timed(torch, stream, flush, steps, lambda: gb.gbsbin_fock_execute(p.handle, t, stream))
            d = p.diagnostics(stream)
            tables[name] = t.cpu().numpy()
        kms = d["point_kernel_ms"]
        achieved = pairs * ops[name] / (kms * 1e-3)
        res[name] = {"ms_per_table": ms / steps, "tables_per_s": 1e3 * steps / ms, "kernel_ms": kms,
                     "pairs_per_s": pairs / (kms * 1e-3), "pipe_ops_per_pair": ops[name],
                     "pipe_ops_per_s": achieved, "pipe_peak": peaks[name][0], "pipe_peak_source": peaks[name][1],
                     "pipe_frac": achieved / peaks[name][0], "sum_P": d["sum_P"], "status": d["status"]}
    res["max_abs_diff_fp64_df32"] = float(np.abs(tables["fp64"] - tables["df32"]).max())
    P = tables["df32"]
    means = [float(np.dot(np.arange(P.shape[l]), P.sum(axis=tuple(m for m in range(L) if m != l)))) for l in range(L)]
    exact = (np.abs(fp.T) ** 2) @ fp.photons.astype(np.float64)
    exact_g = [float(exact[fp.bin_of_mode == l].sum()) for l in range(L)]
    res["group_mean_err_df32"] = float(np.max(np.abs(np.array(means) - np.array(exact_g))))
    return {fp.name: res}


def _extra_e3(gb, torch, stream, flush, steps, world):
    """Total photon number of the largest uniform-loss setup of Sec. VIII: M = 256 (n = 512),
    xi = 0.89, eta = 0.36, Haar U, one detector group, N_max = 170: the one-group Hessenberg
    path in pairs of FP32 and in FP64 against the general FP64 LU kernel on the same table."""
    M, Nmax, xi, eta = 256, 170, 0.89, 0.36
    prob = synth.Problem(M, 1, np.full((M, 1), xi), np.sqrt(eta) * synth.haar_unitary(M, np.random.default_rng(61)),
                         np.zeros(M, np.int32), np.array([Nmax], np.int32))
    res = {}
    tables = {}
    for name, precision, tile in (("hessenberg_fp32_pairs", 1, 0), ("hessenberg_fp64", 0, 0),
                                  ("general_lu_fp64", 0, 3)):
        t0 = time.perf_counter()
        with gb.Plan(prob, precision=precision, want_timing=True, tile_override=tile) as p:
            plan_s = time.perf_counter() - t0
            t = torch.empty(p.shape, dtype=torch.float64, device="cuda")
            gb.gbsbin_execute(p.handle, t, stream)
            ms = _timed(torch, stream, flush, steps, lambda: gb.gbsbin_execute(p.handle, t, stream))
            st, d = p.diagnostics(stream)
            tables[name] = t.cpu().numpy()
            res[name] = {"ms_per_table": ms / steps, "point_kernel_ms": d["point_kernel_ms"],
                         "kernel": d["kernel_name"], "plan_create_s": plan_s, "status": st}
    res["max_abs_diff"] = float(np.abs(tables["hessenberg_fp64"] - tables["general_lu_fp64"]).max())
    res["max_abs_diff_pairs"] = float(np.abs(tables["hessenberg_fp32_pairs"] - tables["general_lu_fp64"]).max())
    return {"E3_M256_n512_L1_N170": res}


def _extra_n32(gb, torch, stream, flush, steps, world):
    """M = 16, K = 1, four groups of four detectors, N_l = 8: 6561 points of 32 x 32 matrices.
    FP32 arithmetic (the tree of block eliminations in pairs of FP32), FP64 (the same tree in
    FP64) and the per-point FP32 + refinement warp kernel, with the tree's own work rate."""
    prob = synth.config(1)
    npts = prob.n_points
    res = {}
    for name, prec, tile in (("fp32", 1, 0), ("fp64", 0, 0), ("per_point_fp32_refine", 1, 5)):
        with gb.Plan(prob, precision=prec, want_timing=True, tile_override=tile) as p:
            t = torch.empty(p.shape, dtype=torch.float64, device="cuda")
            for _ in range(5):
                gb.gbsbin_execute(p.handle, t, stream)
            r = _time_plan(gb, torch, p, t, stream, flush, steps, world)
            d = r["diag"]
            ent = {"ms_per_table": r["ms_per_step"], "points_per_s": world * npts * steps / (r["gpu_ms"] * 1e-3),
                   "tables_per_s": world * steps / (r["gpu_ms"] * 1e-3), "point_kernel_ms": r["kernel_ms"],
                   "kernel": d["kernel_name"], "launches_per_table": d["launches"], "steps": steps}
            issued = _issued_work(prob, d, prec == 1)
            if issued:
                ent.update({"issued": issued[0], "issued_rate": issued[1] / (r["kernel_ms"] * 1e-3) / 1e12,
                            "issued_unit": issued[2], "issued_frac":
                            issued[1] / (r["kernel_ms"] * 1e-3) / 1e12 / issued[3]})
            ent["traffic"] = _profiled_traffic(d["kernel_name"])
            res[name] = ent
    return {"M16_K1_L4_N8_n32_6561pts": res}


def _extra_batch(gb, torch, stream, flush, steps, world):
    out = {}
    # 256 uneven problems, one persistent launch per kernel class, autotuned, graph replay
    probs = synth.batch_config()
    npts = sum(p.n_points for p in probs)
    res = {}
    for name, prec in (("fp32_refine", 1), ("fp64", 0)):
        with gb.Batch(probs, precision=prec, autotune=True) as b:
            b.execute(stream)
            s2 = torch.cuda.Stream()
            torch.cuda.synchronize()
            b.capture(s2)
            b.replay(s2)
            s2.synchronize()
            ms = _timed(torch, s2, flush, steps, lambda: b.replay(s2))
            res[name] = {"ms_per_batch": ms / steps, "tables_per_s": world * len(probs) * steps / (ms * 1e-3),
                         "points_per_s": world * npts * steps / (ms * 1e-3)}
    out["batch256_uneven"] = {"problems": len(probs), "grid_points": npts, **res}
    return out


def backward_work(prob, d):
    """Complex multiply-adds of one reverse pass's point work: one n x n Gauss-Jordan inverse
    per evaluated point (n^3), or along the tree (backward_path 2): per parent (combination of
    the first L - 1 axes' roots) the inverse of the leading groups' block (mE^3), U, V, C
    (2 mE^2 mF + mE mF^2) and the assembly's three products (mF^2 mE + mE^2 mF + mE mF^2), per
    evaluated point the last group's mF^3 inverse."""
    n = prob.n
    if d.get("backward_path") != 2:
        return (float(n) ** 3 * d["n_evaluated"], "k_backward_gj (blocked Gauss-Jordan, per point)",
                "n^3 complex multiply-adds per evaluated point (inverse) x 8 flops")
    labels = np.repeat(np.asarray(prob.bin_of_mode), prob.K)
    mF = 2.0 * float(np.sum(labels == prob.L - 1))      # rows: both halves of each mode
    mE = float(n) - mF
    parents = float(np.prod(prob.radix[:-1]))
    per_parent = mE ** 3 + 2 * mE * mE * mF + mE * mF * mF + (mF * mF * mE + mE * mE * mF + mE * mF * mF)
    macs = parents * per_parent + d["n_evaluated"] * mF ** 3
    return (macs, "k_bwdt_parent + k_bwdt_leaf + k_bwdt_assemble (along the tree)",
            "tree complex multiply-adds (parents' inverses and products, leaves' mF^3 inverses) x 8 flops")


def _extra_n200(gb, torch, stream, flush, steps, world):
    """n = 200 (100 modes, two groups of 50, 81 x 81 grid): the negative log-likelihood of a
    count table, forward table + reverse pass to the adjacency adjoints, in FP32 pairs and in
    FP64, timed with CUDA events on the launching stream (gbsbin_backward_device is
    asynchronous), L2 flushed between steps.  The reverse pass's point work (along the tree:
    the parents' inverses and products and the leaves' Schur-complement inverses) is timed by
    the library's own events; its roofline counts its complex multiply-adds (backward_work) x
    8 flops against the derived peak of its pipe, and for the pairs also 64 FP32-pipe
    operations per complex multiply-add against the FP32 issue rate; the rate of the
    per-point formulation's 8 n^3 flops per point is reported beside it.  The host-chained gradient to the
    physical parameters (gbsbin_backward, synchronous) is timed by wall clock beside it."""
    out = {}
    prob = synth.config(4)
    n = prob.n
    issue32 = SMS * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak32 = 2 * issue32
    peak64 = SMS * FP64_FMA_PER_SM_CLK * 2 * SM_MAX_MHZ * 1e6 / 1e12
    rng = np.random.default_rng(0)
    counts = None
    for precision, name in ((1, "fp32_pairs"), (0, "fp64")):
        with gb.Plan(prob, precision=precision, want_backward=True, want_timing=True) as p:
            t = torch.empty(p.shape, dtype=torch.float64, device="cuda")
            S = torch.empty((n, n), dtype=torch.complex128, device="cuda")
            g = torch.empty((n,), dtype=torch.complex128, device="cuda")
            gb.gbsbin_execute(p.handle, t, stream)
            torch.cuda.synchronize()
            if counts is None:
                Pn = np.clip(t.cpu().numpy(), 1e-300, None)
                counts = torch.from_numpy(rng.multinomial(10 ** 6, (Pn / Pn.sum()).reshape(-1))
                                          .reshape(Pn.shape).astype(np.float64)).cuda()
            dLdP = torch.empty_like(t)

            def step():
                gb.gbsbin_execute(p.handle, t, stream)
                with torch.cuda.stream(stream):
                    torch.div(-counts, t, out=dLdP)
                gb.gbsbin_backward_device(p.handle, dLdP, S, g, stream)
            for _ in range(2):
                step()
            ms = _timed(torch, stream, flush, steps, step) / steps
            st, d = p.diagnostics(stream)
            bms = d["backward_kernel_ms"]
            macs, kname, work = backward_work(prob, d)
            peak, pname = (peak32, "derived FP32") if precision else (peak64, "derived FP64")
            ach = 8.0 * macs / (bms * 1e-3) / 1e12
            entry = {"ms_per_forward_backward": ms, "points_per_s": world * prob.n_points / (ms * 1e-3),
                     "backward_kernel_ms": bms, "forward_point_kernel_ms": d["point_kernel_ms"],
                     "kernel": kname, "timer": "CUDA events on the launching stream, L2 flushed",
                     "per_point_equivalent_tflops": 8.0 * n ** 3 * d["n_evaluated"] / (bms * 1e-3) / 1e12,
                     "roofline": {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                                  "frac": ach / peak, "peak_source": pname, "work": work,
                                  "complex_macs": macs}}
            if precision:
                ops = 64.0 * macs / (bms * 1e-3) / 1e12
                entry["issued"] = {"achieved": ops, "peak": issue32, "unit": "T ops/s", "frac": ops / issue32,
                                   "work": "complex multiply-adds x 64 FP32-pipe operations (pairs)"}
            t0 = time.perf_counter()
            wsteps = max(1, steps // 2)
            for _ in range(wsteps):
                gb.gbsbin_execute(p.handle, t, stream)
                with torch.cuda.stream(stream):
                    torch.div(-counts, t, out=dLdP)
                p.backward(dLdP, stream, want=("r", "T"))
            entry["ms_per_forward_backward_host_chain"] = (time.perf_counter() - t0) / wsteps * 1e3
            out[name] = entry
    return {"M100_K1_L2_N80_n200_gradient": out}


def _sources_hash(paths):
    """Hash of the source files a profiled kernel is built from (its own .cu and headers)."""
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()[:16]


def _profiled_traffic(kernel_name):
    """DRAM bytes per launch of the point kernel (per table for the tree's four launches)
    from the committed ncu summary, or None when no summary exists for this kernel or its
    sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tj = json.load(open(path))
    except (OSError, ValueError):
        return None
    entry = tj.get(kernel_name)
    if not entry:
        return None
    try:
        if _sources_hash(entry["sources"]) != entry["sources_hash"]:
            return None
    except (OSError, KeyError):
        return None
    return entry.get("dram_bytes_per_launch", entry.get("dram_bytes_per_table"))


def cpu_baseline(prob, seconds, tables):
    """The oracle as it stands, whole tables on all host cores, for ~`seconds`; also the
    error of the benchmarked GPU tables against the oracle table."""
    import oracle
    ref = None
    count = 0
    t0 = time.perf_counter()
    while True:
        ref = oracle.binned(prob)["P"]
        count += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    names = {1: "fp32_refine", 0: "fp64", "blk": "per_point_fp32_refine"}
    errs = {names.get(p, str(p)): float(np.abs(tables[p].cpu().numpy() - ref).max()) for p in tables}
    return ({"value": prob.n_points * count / dt, "unit": "points/s", "cores": os.cpu_count(), "kind": "oracle",
             "sample": f"{count} whole {prob.n_points}-point tables in {dt:.1f} s"}, errs)


if __name__ == "__main__":
    sys.exit(main())
