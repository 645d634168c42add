#!/usr/bin/env python3
"""Benchmark of the quasi-particle fRG hot path on GB300.

One step = one flow step of the N_p = 96, 32 x 32 fine-grid workload
(t = 1, t' = 0, mu = 0, U = 2.5, temperature flow from T = 1 with
d ln T = ln 0.98, Z feedback): the two-loop self-energy at xi_j +- 2T and the
Z update, four right-hand-side evaluations (loop kernels + contraction of all
N^3 couplings) and the RK4 combine with the divergence check.  The headline
value is RHS evaluations per second over the timed steps (4 per step, the
self-energy included in the time).  Inputs: synthetic lattice parameters,
no dataset.  All device inputs (partner maps, bubble tables) exceed L2.

The default precision is QPFRG_MIXED_TC (FP32 loop kernels and self-energy,
tensor-core BF16x3 contraction, FP64 state).  The line also carries the
right-hand side alone in the three precisions, self-energy evaluations per
second, and the wall clock of complete flows: the bench workload itself
(full flows/s at N_p = 96) and two small ones (np48_n16 mixed with Z
feedback, np16_n8 FP64 with Z = 1).

--workload sweep128 instead times the 128-flow phase-boundary sweep (N_p in
{24, 48, 72, 96}, 16 x 16 fine grid, Z = 1) through one qpfrg_flow_batch call
and reports complete flows/s (--flows K takes the first K draws).

--impl reference times the FP64 CPU oracle on the host cores (a bounded
sample of output triples per step) for the same metric.
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

WORKLOAD = "np96_n32"
METRIC = "fRG RHS evaluations/s at N_p={N} (flow steps with Z feedback)"
UNIT = "RHS/s"

# Algorithmic work of the method (what any implementation must do), per
# loop-kernel evaluation: ~14 FP32 operations (partner dispersion by angle
# addition, the loop kernel, weight and deposit) + 1 ex2 + 1 reciprocal; per
# self-energy pair: ~20 FP32 operations + 1 ex2 + 1 reciprocal (Fermi factor
# of r) + 2 complex reciprocals (the two chord frequencies, one reciprocal
# each).  The time bound is the slowest pipe: every operation takes one of the
# 128 issue lanes per SM per clock, and the MUFU pipe runs ex2 and rcp at their
# own rates, measured on the device by qpfrg_alu_rates (GB300: ex2 32, rcp 16
# per SM per clock; nominal 16 each where the probe is unavailable).
BUBBLE_FP32_PER_EVAL, BUBBLE_EX2_PER_EVAL, BUBBLE_RCP_PER_EVAL = 14, 1, 1
SIGMA_FP32_PER_PAIR, SIGMA_EX2_PER_PAIR, SIGMA_RCP_PER_PAIR = 20, 1, 3
# issue slots per unit as built: the self-energy's per-pair formula (a packed
# FP32x2 instruction counts one half per pair); the loop kernels' measured
# instructions per computed evaluation on the representative rows of the row
# orbits (ncu smsp__inst_executed x 32 / evaluations at np96_n32:
# 3.29e8 x 32 / 2.27e8)
BUBBLE_ISSUE_AS_BUILT, SIGMA_ISSUE_AS_BUILT = 46.4, 36
# the self-energy pair with its patch read from the patch-of-r table: measured
# instructions per pair (ncu smsp__inst_executed x 32 / pairs at np48_n16:
# 7.03e8 x 32 / 9.06e8)
SIGMA_ISSUE_AS_BUILT_TABLE = 24.8
ISSUE_LANES_PER_SM, NOMINAL_MUFU_PER_SM, N_SM = 128, 16, 152


def alu_clk_per_unit(fp32, ex2, rcp, rates):
    """SM clocks per unit of work at the slowest pipe: the issue lanes, or the
    MUFU pipe at its ex2 and rcp rates (results per SM per clock)."""
    return max((fp32 + ex2 + rcp) / ISSUE_LANES_PER_SM, ex2 / rates["ex2"] + rcp / rates["rcp"])


def alu_rates(api):
    """MUFU rates of this device (qpfrg_alu_rates), else the nominal ones."""
    try:
        r = api.qpfrg_alu_rates()
        return {"ex2": r["ex2"], "rcp": r["rcp"], "ffma": r["ffma"], "source": "measured (qpfrg_alu_rates)"}
    except Exception as e:   # noqa: BLE001 - the figure is informative only
        return {"ex2": NOMINAL_MUFU_PER_SM, "rcp": NOMINAL_MUFU_PER_SM, "ffma": ISSUE_LANES_PER_SM,
                "source": f"nominal ({e})"}


def sigma_units(N, n):
    """(p, q) pairs of one flow-step self-energy launch: the C4v-irreducible
    targets 0..N/8, the mirror-line ones (0, and N/8 when 8 | N) over half of
    the loop points p (the reduced work the kernel does)."""
    M = N * n * n
    mirror = (1.0 if N % 8 == 0 else 0.5) if n % 2 == 0 else 0.0
    return (float(N // 8 + 1) - mirror) * M * M


def bubble_units(N, M, evals_computed=None):
    """Loop-kernel evaluations of one RHS: 2 N^2 M, or the number the library
    reports it computed (a symmetry-reduced launch)."""
    return float(evals_computed) if evals_computed else 2.0 * N * N * M


def cpu_info():
    """Host cores and CPU model of the machine the oracle runs on."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Thread(s) per core", "Socket(s)"):
                info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return info

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the bench workload, valid while the kernel's own source (its
# definition, from the template line to the matching brace) is unchanged: the
# SHA-256 of that text is recorded with the capture; profiles/ holds the summary.
TRAFFIC = {
    # the kernel with its patch-of-r table: DRAM bytes per (p, q) pair from a
    # full capture at np48_n16 (907.7 MB read + 3.3 MB written for 9.06e8
    # pairs: 1.0055 B per pair, the table's byte), scaled to the bench
    # workload's pairs (the table grows with the pairs)
    ("sigma_z", "np96_n32"): {"bytes": 116.61e9, "source": "paper_2005_00827_gb300/csrc/sigma.cu",
                              "kernel": "sigma_fast_kernel", "scaled_from": "np48_n16",
                              "sha256": "85cf7d0d4dc108c73efa7da72ebd52256686955594627914ddebb3dd2bbc19e1"},
}


def kernel_text(path, name):
    """Source of the __global__ function `name` in `path`: from the line before
    its signature (the template line) to the brace that closes its body."""
    src = open(path).read()
    i = src.find(f" {name}(")
    if i < 0:
        return None
    start = src.rfind("\n", 0, src.rfind("\n", 0, i)) + 1
    j = src.find("{", i)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[start:k + 1]
    return None


def traffic_bytes(kernel, workload):
    import hashlib
    t = TRAFFIC.get((kernel, workload))
    if t is None:
        return None
    try:
        text = kernel_text(os.path.join(ROOT, t["source"]), t["kernel"])
    except OSError:
        return None
    if text is None:
        return None
    return t["bytes"] if hashlib.sha256(text.encode()).hexdigest() == t["sha256"] else None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.rows = []
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(local_ms: float, local_units: float, world: int, device=None):
    """Whole-job throughput of independent replicas: units summed over ranks
    divided by the slowest rank's time (max over ranks)."""
    if world == 1:
        return local_units / (local_ms / 1e3), local_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms, local_units], dtype=torch.float64, device=device)
    tmax = t[:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    tsum = t[1:].clone()
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    ms = float(tmax.item())
    return float(tsum.item()) / (ms / 1e3), ms


# ---------------------------------------------------------------------------
def run_qpfrg(args):
    import numpy as np
    import torch

    from paper_2005_00827_gb300 import api, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    wl = inputs.WORKLOADS[args.workload]
    N, n, U = wl["N"], wl["n"], wl["U"]
    prec = {"mixed": api.QPFRG_MIXED, "tc": api.QPFRG_MIXED_TC, "fp64": api.QPFRG_FP64}[args.precision]
    stream = torch.cuda.current_stream()
    ctx = api.Context(N, n, n, U=U, lambda0=1.0, precision=prec, lambda_end=wl["T_end"],
                      z_feedback=int(wl["z_feedback"]), eta=0.02, n_omega=wl["n_omega"], omega_min=-4.0,
                      omega_max=4.0, stream=stream.cuda_stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    # launch shapes measured on this context's own state (untimed)
    tuning = api.qpfrg_autotune(ctx.h, 1.0) if not args.no_autotune else None
    work = api.qpfrg_rhs_work(ctx.h)
    for _ in range(args.warmup):
        api.qpfrg_step(ctx.h, 1)
    barrier()
    api.qpfrg_set_profiling(ctx.h, True)
    api.qpfrg_profile_reset(ctx.h)
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    steps_done = 0
    for _ in range(args.steps):
        r = api.qpfrg_step(ctx.h, 1)
        steps_done += 1
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = api.qpfrg_profile(ctx.h)
    api.qpfrg_set_profiling(ctx.h, False)
    value, ms = aggregate(ms, 4.0 * steps_done, world, device="cuda")
    table_bytes = api.qpfrg_sigma_table(ctx.h)[0]

    # end to end: state uploaded from pinned host memory, one step, state read back
    nbytes = api.qpfrg_state_size(ctx.h)
    img = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    api.qpfrg_get_state_into(ctx.h, img)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        api.qpfrg_set_state_from(ctx.h, img)
        api.qpfrg_step(ctx.h, 1)
        api.qpfrg_get_state_into(ctx.h, img)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": 4.0 * args.steps * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes}

    extra = {}
    # Sigma(k_F, omega) on the workload's frequency grid from the flow's state
    # (one untimed and one timed call; CUDA events on the context's stream)
    if wl["n_omega"] > 0 and not args.no_flows:
        nom = wl["n_omega"]
        Vs = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
        Zs = torch.empty(N, dtype=torch.float64, device="cuda")
        api.qpfrg_read_state(ctx.h, Vs, Zs)
        re = torch.empty(N * nom, dtype=torch.float64, device="cuda")
        im = torch.empty_like(re)
        T_now = float(r.lambda_) if args.steps > 0 else 1.0   # temperature after the timed steps
        api.qpfrg_selfenergy(ctx.h, T_now, Vs, Zs, re, im, None)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        api.qpfrg_selfenergy(ctx.h, T_now, Vs, Zs, re, im, None)
        b.record(stream)
        torch.cuda.synchronize()
        gms = a.elapsed_time(b)
        extra["sigma_grid"] = {"n_omega": nom, "patches": N, "T": T_now, "ms": gms,
                               "evals_per_s": 1e3 / gms}

    # right-hand side alone, mixed and FP64 forms (same inputs)
    V = inputs.random_vertex(N, U, seed=1)
    Z = inputs.z_profile(N, "aniso")
    dV_t = torch.from_numpy(V.ravel()).cuda()
    Z_t = torch.from_numpy(Z).cuda()
    out = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    forms = (("fp64", api.QPFRG_FP64, 3), ("mixed", api.QPFRG_MIXED, 10), ("tc", api.QPFRG_MIXED_TC, 10))
    ref_fp64 = None
    for name, pr, reps in forms:
        with api.Context(N, n, n, U=U, precision=pr, stream=stream.cuda_stream) as c2:
            if tuning is not None:
                api.qpfrg_set_tuning(c2.h, tuning["bubble_qchunk"], tuning["sigma_qblocks"], tuning["tc_splits"], tuning["bubble_transfers"])
            api.qpfrg_rhs(c2.h, 0.1, dV_t, Z_t, out)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                api.qpfrg_rhs(c2.h, 0.1, dV_t, Z_t, out)
            b.record(stream)
            torch.cuda.synchronize()
            extra[f"rhs_only_{name}_per_s"] = reps / (a.elapsed_time(b) / 1e3)
            if pr == api.QPFRG_FP64:
                ref_fp64 = out.clone()
            else:
                # normwise error against the FP64 GPU form on the same inputs
                extra[f"rhs_only_{name}_err_vs_fp64"] = float((out - ref_fp64).abs().max() / ref_fp64.abs().max())
    extra["mixed_vs_fp64_rhs"] = extra["rhs_only_mixed_per_s"] / extra["rhs_only_fp64_per_s"]
    extra["tc_vs_fp64_rhs"] = extra["rhs_only_tc_per_s"] / extra["rhs_only_fp64_per_s"]
    if "sigma_z" in prof and prof["sigma_z"][1] > 0:
        extra["sigma_z_evals_per_s"] = prof["sigma_z"][1] / (prof["sigma_z"][0] / 1e3)

    # complete flows (wall clock of qpfrg_flow, T = 1 down to divergence or T_end)
    if not args.no_flows:
        extra["full_flows"] = [full_flow(api, inputs, "np48_n16", api.QPFRG_MIXED, "mixed", stream),
                               full_flow(api, inputs, "np16_n8", api.QPFRG_FP64, "fp64", stream)]

    # roofline of the dominant kernel (ALU bound: FP32 issue and MUFU pipes)
    peaks, peak_kind = load_peaks()
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kern, key=lambda k: kern[k][0])
    M = N * n * n
    rates = alu_rates(api)
    peak_note = (f"derived: {N_SM} SM x {clk_mhz:.0f} MHz ({peak_kind} sm_max_mhz) x the slower of "
                 f"{ISSUE_LANES_PER_SM} issue lanes per SM per clock (nominal) and the MUFU pipe at "
                 f"ex2 {rates['ex2']:.1f}, rcp {rates['rcp']:.1f} per SM per clock ({rates['source']}; "
                 "MEASURED_PEAKS.json holds no FP32 or MUFU figure)")
    roof = None
    if dom in ("bubble", "sigma_z"):
        if dom == "bubble":
            units = bubble_units(N, M, work["loop_evals"])
            fp32, ex2, rcp = BUBBLE_FP32_PER_EVAL, BUBBLE_EX2_PER_EVAL, BUBBLE_RCP_PER_EVAL
            built = BUBBLE_ISSUE_AS_BUILT
        else:
            units = sigma_units(N, n)
            fp32, ex2, rcp = SIGMA_FP32_PER_PAIR, SIGMA_EX2_PER_PAIR, SIGMA_RCP_PER_PAIR
            built = SIGMA_ISSUE_AS_BUILT_TABLE if table_bytes else SIGMA_ISSUE_AS_BUILT
        peak_units = N_SM * clk_mhz * 1e6 / alu_clk_per_unit(fp32, ex2, rcp, rates)
        avg_s = kern[dom][0] / kern[dom][1] / 1e3
        achieved = units / avg_s
        built_peak = N_SM * clk_mhz * 1e6 * ISSUE_LANES_PER_SM / built
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved / 1e9, "peak": peak_units / 1e9,
                "unit": "Geval/s" if dom == "bubble" else "Gpair/s", "frac": achieved / peak_units,
                "traffic": traffic_bytes(dom, args.workload), "traffic_unit": "bytes per launch",
                "units_per_launch": units, "ms_per_launch": avg_s * 1e3,
                "work_per_unit": f"{fp32} FP32 + {ex2} ex2 + {rcp} rcp (algorithmic)",
                "alu_rates_per_sm_clk": {k: rates[k] for k in ("ex2", "rcp", "ffma")},
                "peak_source": peak_note,
                "issue_efficiency": {"issue_slots_as_built": built, "peak": built_peak / 1e9,
                                     "frac": achieved / built_peak}}

    # the right-hand side's own kernels against their bounds (per RHS of the step)
    rhs_roof = {}
    if "bubble" in kern:
        evals = 2.0 * N * N * M
        red = bubble_units(N, M, work["loop_evals"])
        b_s = kern["bubble"][0] / kern["bubble"][1] / 1e3
        b_peak = N_SM * clk_mhz * 1e6 / alu_clk_per_unit(BUBBLE_FP32_PER_EVAL, BUBBLE_EX2_PER_EVAL,
                                                          BUBBLE_RCP_PER_EVAL, rates)
        rhs_roof["bubble"] = {"bound": "alu", "achieved": red / b_s / 1e9, "peak": b_peak / 1e9, "unit": "Geval/s",
                              "frac": red / b_s / b_peak, "evals_per_rhs": evals, "evals_computed": red,
                              "peak_source": peak_note}
    tc = [k for k in ("tc_fused_pp", "tc_fused_cr", "tc_fused_d") if k in kern]
    if len(tc) == 3:
        # The channel GEMMs stream the FP32 weighted table: pp its pp family
        # (R rows of N^2 floats), cr the ph family, d the ph family twice
        # (K = 2 N^2): 16 R N^2 bytes per RHS, against the HBM copy peak.  On
        # the tensor cores: three BF16 products (hi hi, hi lo, lo hi) of R rows,
        # N columns and K = N^2 (pp, cr) + 2 N^2 (d): 24 R N^3 flop per RHS.
        # R = N^2, or the row orbits of a C4v-symmetric state (their table,
        # written by the loop kernels just before, mostly stays in L2).
        R = float(work.get("contraction_rows") or N * N)
        nbytes, flop = 16.0 * R * N ** 2, 24.0 * R * N ** 3
        t_s = sum(kern[k][0] / kern[k][1] for k in tc) / 1e3
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        rhs_roof["tc_fused"] = {"bound": "hbm", "achieved": nbytes / t_s / 1e9, "peak": hbm, "unit": "GB/s",
                                "frac": nbytes / t_s / 1e9 / hbm, "bytes_per_rhs": nbytes, "ms_per_rhs": t_s * 1e3,
                                "rows": R, "expand_ms_per_rhs": (kern["rows_expand"][0] / kern["rows_expand"][1]
                                                                 if "rows_expand" in kern else 0.0),
                                "peak_source": f"{peak_kind} hbm_gbs",
                                "tensor": {"achieved": flop / t_s / 1e12, "peak": bf16, "unit": "TFLOP/s",
                                           "frac": flop / t_s / 1e12 / bf16, "flop_per_rhs": flop,
                                           "peak_source": f"{peak_kind} bf16_tflops (burst)"}}

    line = {
        "metric": METRIC.format(N=N), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {api.QPFRG_MIXED: "f32+f64", api.QPFRG_MIXED_TC: "bf16x3+f32+f64"}.get(prec, "f64"),
        "data": "synthetic (seeded lattice parameters; no dataset in the paper)",
        "config": {"workload": args.workload, "N_p": N, "fine_grid": f"{n}x{n}", "U": U,
                   "flow": "T-flow from T=1, dlnT=ln0.98, Z feedback, eta=0.02",
                   "precision": args.precision, "l2": "inputs larger than L2 (partner maps "
                   f"{2 * N * N * M / 1e9:.2f} GB, bubble tables)", "parallelism": "replicas",
                   "tuning": tuning},
        "e2e": e2e, "gpu_launches": int(sum(v[1] for v in prof.values())), "rhs_work": work,
        "sigma_table_bytes": table_bytes,
        "kernels_ms": {k: round(v[0], 3) for k, v in kern.items()},
        "kernel_launches": {k: v[1] for k, v in kern.items()},
        "roofline": roof, "rhs_roofline": rhs_roof, "clocks": clk, **extra,
    }
    ctx.close()
    if not args.no_flows:
        # a complete flow of the bench workload itself (fresh context, same shapes)
        line["full_flows"].insert(0, full_flow(api, inputs, args.workload, prec, args.precision, stream, tuning))
    if not args.no_sweep:
        # the 128-flow phase-boundary sweep through one qpfrg_flow_batch call
        line["sweep128"] = sweep128(api, inputs, stream, args)
    if not args.no_shell:
        # energy-shell patching, 32 x 7 = 224 patches
        line["shell224"] = shell224(api, inputs, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_seconds)
        line["cpu_baseline_all_cores"] = cpu_baseline(args.workload, budget_s=args.cpu_seconds,
                                                      nthreads=os.cpu_count() or 1)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def full_flow(api, inputs, workload, prec, name, stream, tuning=None):
    """One complete flow (T = 1 to divergence or T_end): flows/s from the wall clock."""
    import torch
    wl = inputs.WORKLOADS[workload]
    N, n = wl["N"], wl["n"]
    with api.Context(N, n, n, U=wl["U"], lambda0=1.0, precision=prec, lambda_end=wl["T_end"],
                     z_feedback=int(wl["z_feedback"]), eta=0.02, stream=stream.cuda_stream) as c:
        if tuning is not None:
            api.qpfrg_set_tuning(c.h, tuning["bubble_qchunk"], tuning["sigma_qblocks"], tuning["tc_splits"], tuning["bubble_transfers"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = api.qpfrg_flow(c.h)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        d = r.as_dict()
    return {"workload": workload, "precision": name, "flows_per_s": 1.0 / dt, "seconds": dt,
            "steps": d["steps"], "status": d["status"], "lambda_c": d["lambda_c"],
            "z_feedback": bool(wl["z_feedback"])}


# ---------------------------------------------------------------------------
def cpu_baseline(workload, budget_s=15.0, nthreads=1):
    """Oracle RHS on a bounded sample of output triples of the same workload;
    RHS/s = (triples per second) / N^3.  nthreads > 1 runs that many triples at
    once on host threads (the oracle call releases the interpreter lock)."""
    import concurrent.futures as cf

    import numpy as np

    from oracle.oracle import Oracle
    from paper_2005_00827_gb300 import inputs

    wl = inputs.WORKLOADS[workload]
    N, n, U = wl["N"], wl["n"], wl["U"]
    o = Oracle(N, n, n)
    V = inputs.random_vertex(N, U, seed=1)
    Z = inputs.z_profile(N, "aniso")
    nthreads = max(1, int(nthreads))
    stop = time.perf_counter() + budget_s

    def worker(seed):
        rng = np.random.default_rng(seed)
        k = 0
        while time.perf_counter() < stop:
            i, j, l = rng.integers(0, N, 3)
            o.rhs_triple(0.1, V, Z, i, j, l)
            k += 1
        return k

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=nthreads) as ex:
        done = sum(ex.map(worker, range(nthreads)))
    el = time.perf_counter() - t0
    value = done / el / N ** 3
    return {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "host": cpu_info(),
            "sample": f"{done} output triples of the {workload} RHS at T=0.1 in {el:.1f} s on {nthreads} "
                      f"host thread(s) (each triple sums all {N * n * n} loop points in 3 channels); "
                      "RHS/s = triples/s / N^3"}


def sweep128(api, inputs, stream, args):
    """The 128-flow phase-boundary sweep (N_p in {24,48,72,96}, 16 x 16 fine
    grid, Z = 1, seeded draws) through one qpfrg_flow_batch call: complete
    flows/s by CUDA events on the caller's stream (the call returns with its
    work done), the flow steps and the outcomes."""
    import torch
    prec = {"mixed": api.QPFRG_MIXED, "tc": api.QPFRG_MIXED_TC, "fp64": api.QPFRG_FP64}[args.sweep_precision]
    specs = [(d["N"], d["U"], 1.0, d["T_end"]) for d in inputs.batch_specs(128)][:args.flows]
    o = api.qpfrg_default_options()
    o.precision = prec
    o.autotune = 0 if args.no_autotune else 1
    lat, grid = api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(16, 16, 0)
    api.qpfrg_flow_batch(lat, grid, api.QPFRG_REG_TEMPERATURE, o,
                         [(N, 2.0, 1.0, 0.9) for N in (24, 48, 72, 96)], stream.cuda_stream)   # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = api.qpfrg_flow_batch(lat, grid, api.QPFRG_REG_TEMPERATURE, o, specs, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    steps = sum(r["steps"] for r in res)
    status = {}
    for r in res:
        status[r["status"]] = status.get(r["status"], 0) + 1
    return {"flows": len(specs), "flows_per_s": len(specs) / (ms / 1e3), "seconds": ms / 1e3,
            "flow_steps": steps, "rhs_per_s": 4.0 * steps / (ms / 1e3), "statuses": status,
            "precision": args.sweep_precision, "fine_grid": "16x16", "N_p": "24/48/72/96",
            "flow": "T-flow from T=1 to T_end or |V|>20, dlnT=ln0.98, Z=1"}


def shell224(api, inputs, stream):
    """Energy-shell patching (32 angular sections x 7 shells = 224 patches,
    8 x 8 fine points per patch, tensor-core precision): right-hand sides/s,
    one Z evaluation (C4v-irreducible targets) and Z-feedback flow steps/s,
    all by CUDA events on the caller's stream."""
    import torch
    wl = inputs.WORKLOADS["np224_s7"]
    N, n, U, ns = wl["N"], wl["n"], wl["U"], wl["n_shell"]
    kw = dict(U=U, lambda0=1.0, precision=api.QPFRG_MIXED_TC, mode=api.QPFRG_GRID_SHELL, n_shell=ns,
              lambda_end=wl["T_end"], z_feedback=1, eta=0.02, stream=stream.cuda_stream)
    V = torch.from_numpy(inputs.random_vertex(N, U, seed=1, n_shell=ns).ravel()).cuda()
    Z = torch.from_numpy(inputs.z_profile(N, "aniso", n_shell=ns)).cuda()
    out, zo = torch.empty(N ** 3, dtype=torch.float64, device="cuda"), torch.empty(N, dtype=torch.float64,
                                                                                   device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {"workload": "np224_s7", "N_p": N, "shells": ns, "fine_grid": f"{n}x{n} per patch",
           "precision": "tc"}
    with api.Context(N, n, n, **kw) as c:
        api.qpfrg_rhs(c.h, 0.1, V, Z, out)
        api.qpfrg_selfenergy(c.h, 0.1, V, Z, None, None, zo)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(3):
            api.qpfrg_rhs(c.h, 0.1, V, Z, out)
        b.record(stream)
        torch.cuda.synchronize()
        res["rhs_per_s"] = 3 / (a.elapsed_time(b) / 1e3)
        a.record(stream)
        api.qpfrg_selfenergy(c.h, 0.1, V, Z, None, None, zo)
        b.record(stream)
        torch.cuda.synchronize()
        res["sigma_z_ms_all_patches"] = a.elapsed_time(b)
        api.qpfrg_step(c.h, 1)
        torch.cuda.synchronize()
        a.record(stream)
        api.qpfrg_step(c.h, 3)
        b.record(stream)
        torch.cuda.synchronize()
        res["flow_steps_per_s"] = 3 / (a.elapsed_time(b) / 1e3)
        res["flow_rhs_per_s"] = 4 * res["flow_steps_per_s"]
    return res


def run_fig4(args):
    """The comparison grid of Fig. 4 (Sec. 3.2) as our own curves: the
    crossover scale U*(T) of the interaction flow at fixed T (U* = g_c^2 U,
    g_c where the largest coupling first exceeds 100 U, the paper's
    criterion), for the particle-hole channels alone, the full one-loop flow,
    self-energy feedback through the single-scale propagator (the Sigma ODE
    with Z feedback) and the Katanin-corrected flow; 48 angular patches (8 x 8
    fine points per patch) and 32 x 7 = 224 energy-shell patches (4 x 4 fine
    points per patch).  Prints its own line."""
    import time

    import torch

    from paper_2005_00827_gb300 import api

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    U, dg, g_end = 1.0, 0.05, 6.0
    temps = (0.1, 0.15, 0.2, 0.3)
    prec = {"mixed": api.QPFRG_MIXED, "tc": api.QPFRG_MIXED_TC, "fp64": api.QPFRG_FP64}[args.precision]
    variants = {
        "ph_only": dict(channel_mask=api.QPFRG_CH_CR | api.QPFRG_CH_D),
        "one_loop": dict(),
        "s_feedback": dict(sigma_ode=1, z_feedback=1),
        "katanin": dict(sigma_ode=1, z_feedback=1, katanin=1),
    }
    grids = {"np48": dict(N=48, n=8), "np224_s7": dict(N=224, n=4, mode=api.QPFRG_GRID_SHELL, n_shell=7)}
    t0 = time.time()
    curves = {}
    for gname, gkw in grids.items():
        for vname, vkw in variants.items():
            pts = []
            for T in temps:
                kw = dict(gkw)
                N, n = kw.pop("N"), kw.pop("n")
                with api.Context(N, n, n, U=U, lambda0=0.0, regulator=api.QPFRG_REG_INTERACTION, T_fixed=T,
                                 eta=0.05, step=dg, lambda_end=g_end, stop_abs_v=100.0 * U,
                                 precision=prec, stream=stream.cuda_stream, **kw, **vkw) as c:
                    r = api.qpfrg_flow(c.h).as_dict()
                pts.append({"T": T, "status": r["status"], "g_c": r["lambda_c"] if r["status"] == "DIVERGED" else None,
                            "U_star": r["lambda_c"] ** 2 * U if r["status"] == "DIVERGED" else None,
                            "steps": r["steps"]})
            curves[f"{vname}@{gname}"] = pts
    print(json.dumps({"mode": "fig4", "criterion": "max|V| > 100 U, U* = g_c^2 U", "U": U, "dg": dg,
                      "precision": args.precision, "curves": curves, "seconds": time.time() - t0}))


def run_sweep(args):
    """The 128-flow phase-boundary sweep (N_p in {24,48,72,96}, 16 x 16 fine
    grid, Z = 1, seeded draws) through qpfrg_flow_batch: complete flows/s."""
    import torch

    from paper_2005_00827_gb300 import api, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    prec = {"mixed": api.QPFRG_MIXED, "tc": api.QPFRG_MIXED_TC, "fp64": api.QPFRG_FP64}[args.precision]
    n = 16
    specs = [(d["N"], d["U"], 1.0, d["T_end"]) for d in inputs.batch_specs(128)][:args.flows]
    stream = torch.cuda.current_stream()
    o = api.qpfrg_default_options()
    o.precision = prec
    o.autotune = 0 if args.no_autotune else 1     # shapes per patch-count group
    lat, grid = api.qpfrg_lattice(1.0, 0.0, 0.0), api.qpfrg_fine_grid(n, n, 0)
    for _ in range(args.warmup):   # one short flow per patch count
        api.qpfrg_flow_batch(lat, grid, api.QPFRG_REG_TEMPERATURE, o,
                             [(N, 2.0, 1.0, 0.9) for N in (24, 48, 72, 96)], stream.cuda_stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    res = api.qpfrg_flow_batch(lat, grid, api.QPFRG_REG_TEMPERATURE, o, specs, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value, ms = aggregate(ms, float(len(specs)), world, device="cuda")
    steps = sum(r["steps"] for r in res)
    status = {}
    for r in res:
        status[r["status"]] = status.get(r["status"], 0) + 1
    line = {"metric": "complete fRG flows/s (phase-boundary sweep, one batched call)", "value": value,
            "unit": "flows/s", "n_gpus": world, "steps": 1, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {api.QPFRG_MIXED: "f32+f64", api.QPFRG_MIXED_TC: "bf16x3+f32+f64"}.get(prec, "f64"),
            "data": "synthetic (seeded parameter draws, splitmix64 seed 20050082)",
            "config": {"workload": "sweep128", "flows": len(specs), "N_p": "24/48/72/96", "fine_grid": "16x16",
                       "autotune": not args.no_autotune,
                       "flow": "T-flow from T=1 to T_end or |V|>20, dlnT=ln0.98, Z=1",
                       "precision": args.precision, "parallelism": "replicas"},
            "flow_steps": steps, "rhs_per_s": 4.0 * steps / (ms / 1e3), "statuses": status, "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def run_reference(args):
    from paper_2005_00827_gb300 import inputs

    rank, world, _ = dist_env()
    if rank != 0:
        return
    budget = max(1.0, args.cpu_seconds / max(1, args.steps))
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(args.workload, budget_s=0.5)
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.workload, budget_s=budget)["value"])
    v = statistics.mean(vals)
    cb = cpu_baseline(args.workload, budget_s=1.0)
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC.format(N=inputs.WORKLOADS[args.workload]["N"]), "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 4e3 / v,
            "ms_per_step_kind": "extrapolated: one step is 4 RHS of N^3 triples; each timed step runs "
                                f"{budget:.1f} s on a sample of triples and scales by N^3 / triples done",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_rhs_only(args):
    """One context of the workload at one precision, right-hand sides only
    (Z feedback off, fixed seeded vertex): the small single-context command
    that kernel captures run under.  Prints its own JSON line (not a bench
    line): RHS/s over the timed calls and the per-kernel profile."""
    import torch

    from paper_2005_00827_gb300 import api, inputs

    torch.cuda.set_device(0)
    wl = inputs.WORKLOADS[args.workload]
    N, n, U = wl["N"], wl["n"], wl["U"]
    ns = wl.get("n_shell", 1)
    mode = api.QPFRG_GRID_SHELL if ns > 1 else api.QPFRG_GRID_WEDGE
    prec = {"mixed": api.QPFRG_MIXED, "tc": api.QPFRG_MIXED_TC, "fp64": api.QPFRG_FP64}[args.rhs_only]
    stream = torch.cuda.current_stream()
    V = torch.from_numpy(inputs.random_vertex(N, U, seed=1, n_shell=ns).ravel()).cuda()
    Z = torch.from_numpy(inputs.z_profile(N, "aniso", n_shell=ns)).cuda()
    out = torch.empty(N ** 3, dtype=torch.float64, device="cuda")
    tuning = None
    with api.Context(N, n, n, U=U, precision=prec, mode=mode, n_shell=ns, stream=stream.cuda_stream) as c:
        if args.tune:
            tuning = api.qpfrg_autotune(c.h, args.lam)
        elif args.bubble_transfers:
            api.qpfrg_set_tuning(c.h, bubble_transfers=args.bubble_transfers)
        for _ in range(args.warmup):
            api.qpfrg_rhs(c.h, args.lam, V, Z, out)
        torch.cuda.synchronize()
        api.qpfrg_set_profiling(c.h, True)
        api.qpfrg_profile_reset(c.h)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            api.qpfrg_rhs(c.h, args.lam, V, Z, out)
        b.record(stream)
        torch.cuda.synchronize()
        prof = api.qpfrg_profile(c.h)
        ms = a.elapsed_time(b)
        sig_ms = None
        if args.sigma:
            # one evaluation of Z on every patch (chord about xi_j), after an untimed one
            api.qpfrg_set_profiling(c.h, False)
            zo = torch.empty(N, dtype=torch.float64, device="cuda")
            api.qpfrg_selfenergy(c.h, 0.1, V, Z, None, None, zo)
            a.record(stream)
            api.qpfrg_selfenergy(c.h, 0.1, V, Z, None, None, zo)
            b.record(stream)
            torch.cuda.synchronize()
            sig_ms = a.elapsed_time(b)
    print(json.dumps({"mode": "rhs_only", "workload": args.workload, "precision": args.rhs_only, "T": args.lam,
                      "rhs_per_s": args.steps / (ms / 1e3), "ms_per_rhs": ms / args.steps,
                      "kernels_ms_per_rhs": {k: v[0] / args.steps for k, v in prof.items() if v[1] > 0},
                      "launches": {k: v[1] for k, v in prof.items() if v[1] > 0},
                      "sigma_z_ms": sig_ms, "tuning": tuning, "bubble_transfers": args.bubble_transfers}))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="qpfrg", choices=["qpfrg", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--precision", default="tc", choices=["mixed", "tc", "fp64"])
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-flows", action="store_true", help="skip the complete-flow timings")
    p.add_argument("--flows", type=int, default=128, help="sweep128: number of flows (first of the draws)")
    p.add_argument("--no-autotune", action="store_true", help="built-in launch shapes instead of qpfrg_autotune")
    p.add_argument("--no-sweep", action="store_true", help="skip the 128-flow sweep summary of the default line")
    p.add_argument("--sweep-precision", default="tc", choices=["mixed", "tc", "fp64"])
    p.add_argument("--no-shell", action="store_true", help="skip the energy-shell summary of the default line")
    p.add_argument("--rhs-only", choices=["mixed", "tc", "fp64"],
                   help="time right-hand sides of one context only (kernel captures); prints its own line")
    p.add_argument("--sigma", action="store_true", help="--rhs-only: also time one Z evaluation")
    p.add_argument("--tune", action="store_true", help="--rhs-only: qpfrg_autotune the context first")
    p.add_argument("--lam", type=float, default=0.1, help="--rhs-only: temperature of the right-hand sides")
    p.add_argument("--bubble-transfers", type=int, default=0, choices=[0, 2, 4],
                   help="--rhs-only: transfers per warp pass of the loop kernels (0: built-in)")
    args = p.parse_args()
    if args.warmup < 3 and args.impl == "qpfrg":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.rhs_only:
        run_rhs_only(args)
    elif args.workload == "fig4":
        run_fig4(args)
    elif args.workload == "sweep128":
        run_sweep(args)
    else:
        run_qpfrg(args)


if __name__ == "__main__":
    main()
