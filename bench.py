"""Benchmark: inverse-DFT iterations per second on one B300 (and replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cube32_q4_e100] [--prec mixed|fp64]

A step is one full inverse iteration through the C ABI (invdft_step): the
L-BFGS direction, a backtracking line search (one Kohn-Sham solve by
Chebyshev-filtered subspace iteration per trial), the loss, the batched
projected MINRES adjoint solves for every occupied orbital and the gradient
reduction, with the paper's adaptive tolerances (c_eig = 1e2, c_ad = 1e5,
tau_BC = 1e-6).  The default workload is the 100-electron, 32^3-cell Q4 case
(2,048,383 unknowns, 60 states, 50 adjoint columns); the target density is
generated at set-up by a Kohn-Sham solve at a known reference potential (the
paper's molecular densities are not available).  Every orbital block is
larger than L2 (0.98 GB in FP64), so no flush is needed between steps.

The JSON line also carries the operator benchmark of the same mesh
(H~X on 64 vectors, nominal 2 (p+1)^6 N_v n_cells flops), the roofline of the
dominant kernel (H~X, timed with CUDA events inside the timed steps), the
oracle as a CPU baseline, an end-to-end figure through host buffers and the
SM clocks sampled during the timed region.

Multi-GPU: the path runs as independent replicas (one problem per rank, no
collective in the data path); value = steps of all ranks / max rank time.
--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "inverse-DFT iterations/s (mixed FP32/TF32 + FP64 GPU path)"

# DRAM bytes per (node, column) of one FP32 CUDA-core H~X launch: ncu
# dram__bytes_read.sum + dram__bytes_write.sum of hx_simt_kernel<64, 0> (TMA
# brick version) on the 24^3-cell Q4 mesh (857,375 unknowns) with 60 columns,
# 486.90 + 190.83 MB, plus the 4-byte zero fill of Z that precedes the kernel
# in the same launch.  Traffic grows with unknowns x columns, so the in-step
# figure scales by them.
HX_SIMT_DRAM_BYTES_PER_NODE_COL = (486.90e6 + 190.83e6) / (857375 * 60) + 4.0

# H~X column-applications per inverse iteration on each workload, as counted by
# the GPU path (line-search solves, Chebyshev passes, MINRES iterations) over the
# timed steps of a mixed-precision run (cube32_q4_e100: 32,750 on average over
# three steps; the smaller workloads carry estimates from their Chebyshev
# pass and MINRES iteration counts).  The reference arm uses these fixed
# counts so that it never touches the GPU.
COL_APPLIES_PER_STEP = {"cube32_q4_e100": 32750,
                        "cube24_q4_e20": 16 * 31 * 3 + 10 * 200,
                        "cube8_q2_he": 8 * 21 * 3 + 100, "cube32_q4_hx": 64}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cube32_q4_e100",
                    choices=sorted(W.WORKLOADS) + ["batch16"],
                    help="batch16: the sixteen small problems stepped as one batch")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-hx", action="store_true", help="skip the operator benchmark")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ncell", type=int, default=None,
                    help="run the workload on NCELL^3 cells of the same box (a smaller case "
                         "for kernel profiles; the printed line then names that mesh)")
    ap.add_argument("--hx-case", nargs=3, metavar=("NCELL", "NCOL", "KIND"), default=None,
                    help="only apply H~X three times on an NCELL^3 Q4 mesh with NCOL random "
                         "columns, KIND tf32|fp32|fp64 (a small case for kernel profiles)")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons every 200 ms (read only)."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ problem set-up

def build_problem(wl, prec, device):
    import torch

    import paper_2510_10529_b300 as P
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                   kT=wl.kT, prec=prec, cheb_degree=wl.cheb_degree, seed=wl.seed + 1,
                   device=device)
    xyz = pb.coords()
    f = W.model_fields(wl, xyz)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
    v_fixed, v_ref = t(f["v_fixed"]), t(f["v_xc_ref"])
    # target density: a tight Kohn-Sham solve at the reference potential
    gen = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                    kT=wl.kT, prec="mixed", cheb_degree=wl.cheb_degree, eig_tol=1e-9,
                    seed=wl.seed + 2, device=device)
    gen.set_potential(v_fixed, v_ref)
    rho_data = gen.forward_solve()["rho"].clone()
    gen.close()
    del gen
    torch.cuda.empty_cache()
    pb.set_potential(v_fixed, None)
    return pb, dict(v_fixed=v_fixed, v_ref=v_ref, rho_data=rho_data,
                    w=torch.ones(pb.L, dtype=torch.float64, device=device))


def hx_benchmark(device, reps32=20, reps64=3):
    """H~X on the 32^3-cell Q4 operator benchmark (64 unit-norm random vectors)."""
    import torch

    import paper_2510_10529_b300 as P
    wl = W.cube32_q4_hx()
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, nstates=8, device=device)
    xyz = pb.coords()
    v = W.smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
    pb.set_potential(torch.as_tensor(v, dtype=torch.float64, device=device))
    X64 = torch.as_tensor(W.random_block(pb.L, 64, wl.seed), device=device)
    out = {}
    ne, cells = (wl.order + 1) ** 3, wl.ncell ** 3
    flops = 2.0 * ne * ne * 64 * cells
    for name, X, reps, tc in (("mixed", X64.float(), reps32, True),
                              ("fp32", X64.float(), reps32, False), ("fp64", X64, reps64, False)):
        Y = torch.empty_like(X)
        for _ in range(3):
            P.invdft_apply_h(pb.h, X, Y, tc)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            P.invdft_apply_h(pb.h, X, Y, tc)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        byt = (2 * 64 * X.element_size() + 8) * pb.L
        out[name] = {"ms": ms, "tflops_nominal": flops / ms / 1e9, "gbs": byt / ms / 1e6}
    pb.close()
    return {"workload": "cube32_q4_hx", "ncol": 64, "nominal_flops": flops, **out}


def hx_case(ncell, ncol, kind, device):
    """Three H~X applications on an ncell^3 Q4 mesh of the operator-benchmark box
    (a small case that a kernel profiler can capture in seconds)."""
    import torch

    import paper_2510_10529_b300 as P
    wl = W.cube32_q4_hx()
    pb = P.Problem(wl.lo, wl.hi, ncell, 4, nstates=8, device=device)
    xyz = pb.coords()
    v = W.smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
    pb.set_potential(torch.as_tensor(v, dtype=torch.float64, device=device))
    X = torch.as_tensor(W.random_block(pb.L, ncol, wl.seed), device=device)
    if kind != "fp64":
        X = X.float()
    Y = torch.empty_like(X)
    for _ in range(3):
        P.invdft_apply_h(pb.h, X, Y, kind == "tf32")
    torch.cuda.synchronize()
    pb.close()
    print(json.dumps({"hx_case": {"ncell": ncell, "unknowns": pb.L, "ncol": ncol, "kind": kind}}))


# ------------------------------------------------------------------ oracle baseline

def oracle_baseline(wl, col_applies_per_step: float, budget_s: float = 12.0):
    """Time the oracle's H~X (numpy FP64 cell loop) on the full mesh with a few
    columns, and scale to the column-applications of one GPU step."""
    from oracle import fe
    try:
        from threadpoolctl import threadpool_info
        cores = max([t.get("num_threads", 1) for t in threadpool_info()] or [1])
    except Exception:
        cores = 1
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    ncol = 2
    X = W.random_block(mesh.L, ncol, wl.seed)
    v = np.zeros(mesh.L)
    t0 = time.perf_counter()
    reps = 0
    while True:
        mesh.apply_Htilde(v, X)
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 8:
            break
    per_col = (time.perf_counter() - t0) / (reps * ncol)
    step_s = per_col * col_applies_per_step
    return {"value": 1.0 / step_s, "unit": "iter/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle H~X (numpy FP64 cell loop, {wl.name} mesh, {ncol} columns, "
                       f"{reps} applications, {per_col:.3f} s per column) x "
                       f"{col_applies_per_step:.0f} column-applications per step; a lower "
                       "bound on the oracle's time per iteration (its Gram, eigensolver and "
                       "MINRES vector work are not counted)")}


# ------------------------------------------------------------------ arms

def workload_of(args):
    wl = W.WORKLOADS[args.workload]()
    if args.ncell:
        wl = dataclasses.replace(wl, ncell=args.ncell)
    return wl


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest value of x over the ranks (all ranks call it; x itself
    when world == 1)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds_max


def run_ours(args, rank, world):
    import torch
    import torch.distributed as dist

    import paper_2510_10529_b300 as P
    local = int(os.environ.get("LOCAL_RANK", "0"))
    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    wl = workload_of(args)
    pb, d = build_problem(wl, args.prec, device)
    v_xc = torch.zeros(pb.L, dtype=torch.float64, device=device)
    rd, w = d["rho_data"], d["w"]
    for _ in range(args.warmup):
        pb.step(rd, w, v_xc)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    pb.profile_hx(True)
    launches0 = P.invdft_kernel_launches()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # INVDFT_PROFILE_TIMED=1 brackets the timed steps for a profiler started
    # with capture off (ncu --profile-from-start off); it changes no work
    profile_timed = os.environ.get("INVDFT_PROFILE_TIMED") == "1"
    if profile_timed:
        torch.cuda.profiler.start()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(pb.step(rd, w, v_xc))
    e1.record(stream)
    torch.cuda.synchronize()
    if profile_timed:
        torch.cuda.profiler.stop()
    launches = P.invdft_kernel_launches() - launches0
    prof = pb.profile_hx(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, world, device)
    if world > 1:
        dist.barrier()
    value = whole_job_rate(1.0, world, ms_max / 1e3)

    # end to end through host buffers: v_xc pinned on the host, copied in and
    # out every step, plus the loss read back
    v_host = v_xc.cpu().pin_memory()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        v_dev = v_host.to(device, non_blocking=True)
        pb.step(rd, w, v_dev)
        v_host.copy_(v_dev, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world, device)
    e2e = {"value": whole_job_rate(1.0, world, e2e_s), "unit": "iter/s",
           "h2d_bytes_per_step": pb.L * 8, "d2h_bytes_per_step": pb.L * 8 + 8}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return
    hx = None if args.no_hx else hx_benchmark(device)
    pk = peaks()
    simt = prof["fp32"]["launches"] > 0
    k32 = prof["fp32"] if simt else prof["fp64"]
    nl = max(1, k32["launches"])
    achieved = k32["bytes"] / (k32["ms"] * 1e6) if k32["ms"] > 0 else None
    peak_gbs = pk["hbm_gbs"] if pk else 6400.0
    ne, cells = (wl.order + 1) ** 3, wl.ncell ** 3
    col_applies = sum(prof[k]["flops"] for k in ("fp64", "fp32", "tf32")) / (2.0 * ne * ne * cells)
    bytes_per_launch = k32["bytes"] / nl
    traffic = None
    if simt:
        ncol_avg = (bytes_per_launch / pb.L - 4.0) / 8.0
        traffic = HX_SIMT_DRAM_BYTES_PER_NODE_COL * pb.L * ncol_avg
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
            "frac": (achieved / peak_gbs) if achieved else None, "traffic": traffic,
            "kernel": ("hx_simt_kernel: FP32 H~X of the MINRES iterations (CUDA cores)" if simt
                       else "hx_cells + hx_nodal: FP64 H~X"),
            "launches": int(k32["launches"]), "avg_launch_ms": k32["ms"] / nl,
            "peak_source": "measured" if pk else "fallback",
            "algorithmic_bytes_per_launch": bytes_per_launch}
    cpu = None
    if not args.no_cpu:
        cpu = oracle_baseline(wl, col_applies / args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": wl.name, "cells": f"{wl.ncell}^3", "order": wl.order,
                   "unknowns": pb.L, "nstates": wl.nstates, "n_electrons": wl.n_electrons,
                   "prec": args.prec, "cheb_degree": wl.cheb_degree,
                   "l2": "inputs larger than L2 (orbital blocks 0.98 GB FP64), no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clk, "hx": hx,
        "step_stats": {"loss_last": stats[-1]["loss"], "err_l2_last": stats[-1]["err_l2"],
                       "cheb_passes": [s["cheb_passes"] for s in stats],
                       "minres_iters": [s["minres_iters_max"] for s in stats],
                       "ls_trials": [s["ls_trials"] for s in stats],
                       # host wall time of the forward solves (all line-search
                       # trials) and of the adjoint solve of each step
                       "t_forward_ms": [s["t_forward_ms"] for s in stats],
                       "t_adjoint_ms": [s["t_adjoint_ms"] for s in stats],
                       "col_applies_per_step": col_applies / args.steps,
                       "hx_ms_share": sum(prof[k]["ms"] for k in ("fp64", "fp32", "tf32"))
                       / (ms_max * args.steps),
                       "hx_fp64_ms_per_step": prof["fp64"]["ms"] / args.steps,
                       "hx_fp32_ms_per_step": prof["fp32"]["ms"] / args.steps,
                       "hx_tf32_ms_per_step": prof["tf32"]["ms"] / args.steps},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args, rank, world):
    """Sixteen small problems (workloads.batch16) stepped as one batch: their
    Chebyshev filter passes run as single persistent launches while each
    problem's other work runs on its own stream; timed against the same
    problems stepped one after another."""
    import torch

    import paper_2510_10529_b300 as P
    local = int(os.environ.get("LOCAL_RANK", "0"))
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    wls = W.batch16()
    built = [build_problem(wl, "mixed", device) for wl in wls]
    rd = [d["rho_data"] for _, d in built]
    w = [d["w"] for _, d in built]

    def fresh():
        out = []
        for wl, (pb0, d) in zip(wls, built):
            pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates,
                           n_electrons=wl.n_electrons, kT=wl.kT, prec="mixed",
                           cheb_degree=wl.cheb_degree, seed=wl.seed + 1, device=device)
            pb.set_potential(d["v_fixed"], None)
            out.append(pb)
        return out

    def zeros(pbs):
        return [torch.zeros(pb.L, dtype=torch.float64, device=device) for pb in pbs]

    # one after another
    seq = fresh()
    v_seq = zeros(seq)
    for _ in range(args.warmup):
        for b, pb in enumerate(seq):
            pb.step(rd[b], w[b], v_seq[b])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for b, pb in enumerate(seq):
            pb.step(rd[b], w[b], v_seq[b])
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) / args.steps
    for pb in seq:
        pb.close()
    # batched
    probs = fresh()
    v_b = zeros(probs)
    batch = P.Batch(probs)
    for _ in range(args.warmup):
        batch.step(rd, w, v_b)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = P.invdft_kernel_launches()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(batch.step(rd, w, v_b)[0])
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = P.invdft_kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / args.steps
    n = len(wls)
    line = {
        "metric": "batched inverse-DFT problem-iterations/s (16 small problems, one batch)",
        "value": n / (ms / 1e3), "unit": "problem-iter/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "batch16", "problems": n,
                   "cells": [f"{wl.ncell}^3 Q{wl.order}" for wl in wls],
                   "n_electrons": [wl.n_electrons for wl in wls],
                   "nstates": [wl.nstates for wl in wls], "cheb_degree": wls[0].cheb_degree,
                   "l2": "working sets below L2 size (small problems), no flush",
                   "parallelism": "one batch"},
        "sequential": {"value": n / t_seq, "unit": "problem-iter/s",
                       "ms_per_step": t_seq * 1e3},
        "batch": batch.info(), "graphs": P.invdft_graph_stats(), "gpu_launches": int(launches),
        "clocks": clk,
        "final_err_l2": [s["err_l2"] for s in stats[-1]],
    }
    batch.close()
    print(json.dumps(line), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]()
    per_step = COL_APPLIES_PER_STEP[wl.name]
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(oracle_baseline(wl, per_step, budget_s=4.0))
    vals = vals[args.warmup:]
    v = statistics.median([x["value"] for x in vals])
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "cells": f"{wl.ncell}^3", "order": wl.order,
                       "unknowns": wl.n_interior, "nstates": wl.nstates,
                       "n_electrons": wl.n_electrons, "parallelism": "cpu"},
            "cpu_baseline": {**vals[-1], "value": v},
            "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.hx_case:
        n, k, kind = args.hx_case
        if kind not in ("tf32", "fp32", "fp64"):
            raise SystemExit("--hx-case KIND must be tf32, fp32 or fp64")
        hx_case(int(n), int(k), kind, "cuda")
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload == "batch16":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "the batched workload has no oracle arm; see the default workload"}))
        elif rank == 0:
            run_batch(args, rank, world)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
