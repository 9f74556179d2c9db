"""Benchmark: inverse-DFT iterations per second on one B300 (and replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload cube32_q4_e100] [--prec mixed|fp64] [--fp64-steps K64]

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

Timed steps: each of the K timed steps copies v_xc in from pinned host memory,
runs invdft_step and copies v_xc and the loss back.  `value` is the device
time of the steps alone (CUDA events around each invdft_step call on its
stream); `e2e` is the host wall time of the same steps including both copies.

Headline comparison (the metric's "mixed vs FP64 GPU path at equal
accuracy"): after the mixed arm, the plain FP64 GPU path runs the same
trajectory from the same start for K64 steps (1 untimed + K64 - 1 timed by
default, fewer than the mixed arm because an FP64 step takes tens of
seconds); the line reports both iteration rates, the e_L2 of both arms after
every common step, and the relative difference of the two paths' gradients
at the FP64 arm's last iterate.

The JSON line also carries the operator benchmark of the same mesh (H~X on 64
vectors in FP32, TF32 and FP64, nominal 2 (p+1)^6 N_v n_cells flops), the
roofline of the in-step FP32 H~X of the MINRES iterations (CUDA events on its
stream, algorithmic bytes over device time), the in-step filter launches, the
oracle as a CPU baseline and the SM clocks sampled during the timed region.

Multi-GPU: the path runs as independent replicas (one problem per rank, no
collective in the data path); value = steps of all ranks / max rank time.
--impl reference times the FP64 CPU oracle (rank 0 only): each step is one
full oracle iteration of the 8^3-cell Q2 two-electron workload (the large
workload's oracle iteration takes hours; its oracle H~X per column is
measured and reported, its iteration rate is not run).
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

# DRAM bytes per (node, column) of one FP32 sweep-form H~X launch of the MINRES
# kind (plain epilogue, no W / E): ncu dram__bytes_read.sum +
# dram__bytes_write.sum of hx_sweep_kernel on the 24^3-cell Q4 mesh (857,375
# unknowns) with 60 columns, tile variant 2, z segments of 6 cells
# (profiles/hx_sweep_cube24_q4_60cols.md): 245,347,328 + 170,093,312 bytes.
HX_SWEEP_DRAM_BYTES_PER_NODE_COL = (245464832 + 169656832) / (857375 * 60)
HX_SWEEP_DRAM_SOURCE = "profiles/hx_sweep_cube24_q4_60cols.md"

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
    ap.add_argument("--fp64-steps", type=int, default=3,
                    help="steps of the FP64 comparison arm (the first one untimed); 0 skips it")
    ap.add_argument("--no-hx", action="store_true", help="skip the operator benchmark")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ncell", type=int, default=None,
                    help="run the workload on NCELL^3 cells of the same box (a smaller case "
                         "for kernel profiles; the printed line then names that mesh)")
    ap.add_argument("--hx-variant", type=int, default=-1,
                    help="with --hx-case: fix the sweep kernel's tile variant (-1: autotuned)")
    ap.add_argument("--hx-seglen", type=int, default=0,
                    help="with --hx-case: fix the sweep kernel's z-segment length (0: autotuned)")
    ap.add_argument("--oracle-iterations", nargs=2, metavar=("BUDGET_S", "MAX"), default=None,
                    help=argparse.SUPPRESS)
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


def _schedule(vs):
    """(variant, seglen) of the sweep H~X with the balanced schedule named."""
    from paper_2510_10529_b300 import INVDFT_HX_SEG_BALANCED
    v, seg = vs
    return [v, "balanced" if seg == INVDFT_HX_SEG_BALANCED else seg]


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


def measured_rates():
    """Arithmetic rates of this device (TFLOP/s) from the library's probes:
    FP64 FMA, FP32 FMA, packed FP32 FMA pairs, TF32 tensor-core MMAs."""
    import paper_2510_10529_b300 as P
    try:
        return {k: P.invdft_peak_probe(k) for k in ("fp64", "fp32", "fp32x2", "tf32")}
    except Exception as exc:      # a probe failure must not lose the bench line
        return {"error": repr(exc)}


def hx_benchmark(device, reps32=50, reps64=50, rates=None):
    """H~X on the 32^3-cell Q4 operator benchmark (64 unit-norm random vectors):
    TF32 tensor cores (dense cell GEMM), FP32 and FP64 sweep form (CUDA cores).
    Each timing is the median over `reps` launches, each between its own pair
    of CUDA events, after 5 warm-up launches (the autotuner's first launch
    among them); the blocks (0.5 GB FP32, 1.05 GB FP64) are larger than L2."""
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
    pk = peaks()
    hbm = pk["hbm_gbs"] if pk else 6400.0
    for name, X, reps, tc in (("tf32", X64.float(), reps32, True),
                              ("fp32", X64.float(), reps32, False), ("fp64", X64, reps64, False)):
        Y = torch.empty_like(X)
        for _ in range(5):
            P.invdft_apply_h(pb.h, X, Y, tc)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(reps)]
        for e0, e1 in ev:
            e0.record()
            P.invdft_apply_h(pb.h, X, Y, tc)
            e1.record()
        torch.cuda.synchronize()
        ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
        # X read, Y written, v read (FP32 copy on the FP32 CUDA-core path)
        vbytes = 4 if name == "fp32" else 8
        byt = (2 * 64 * X.element_size() + vbytes) * pb.L
        out[name] = {"ms": ms, "tflops_nominal": flops / ms / 1e9, "gbs": byt / ms / 1e6,
                     "hbm_frac": byt / ms / 1e6 / hbm, "algorithmic_bytes": byt}
        if name == "fp64" and rates and "fp64" in rates:
            # the FP64 sweep executes about 100 FLOP per (node, column) (the
            # seven even/odd banded sweeps, the partial cells at tile edges and
            # the x halo): its rate against the measured FP64 FMA rate
            ex = 100.0 * pb.L * 64
            out[name]["fp64_pipe"] = {"executed_flops_est": ex, "tflops": ex / ms / 1e9,
                                      "peak_tflops": rates["fp64"],
                                      "frac": ex / ms / 1e9 / rates["fp64"]}
        if name != "tf32":
            out[name]["tuned_variant_seglen"] = _schedule(pb.hx_config(64, name == "fp64")["plain"])
    pb.close()
    return {"workload": "cube32_q4_hx", "ncol": 64, "nominal_flops": flops,
            "peak_gbs": hbm, "peak_source": "measured" if pk else "fallback", **out}


def hx_case(ncell, ncol, kind, device, variant=-1, seglen=0):
    """Three H~X applications on an ncell^3 Q4 mesh of the operator-benchmark box
    (a small case that a kernel profiler can capture in seconds)."""
    import torch

    import paper_2510_10529_b300 as P
    wl = W.cube32_q4_hx()
    pb = P.Problem(wl.lo, wl.hi, ncell, 4, nstates=8, device=device)
    xyz = pb.coords()
    v = W.smeared_coulomb(xyz, wl.nuclei_R, wl.nuclei_Z, wl.smear)
    pb.set_potential(torch.as_tensor(v, dtype=torch.float64, device=device))
    pb.tune_hx(variant, seglen)
    X = torch.as_tensor(W.random_block(pb.L, ncol, wl.seed), device=device)
    if kind != "fp64":
        X = X.float()
    Y = torch.empty_like(X)
    for _ in range(3):
        P.invdft_apply_h(pb.h, X, Y, kind == "tf32")
    torch.cuda.synchronize()
    pb.close()
    print(json.dumps({"hx_case": {"ncell": ncell, "unknowns": pb.L, "ncol": ncol, "kind": kind,
                                  "variant": variant, "seglen": seglen}}))


# ------------------------------------------------------------------ oracle baseline

def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_iterations_here(budget_s: float, max_iters: int):
    """Full oracle iterations (oracle.inverse.step: line search with a Kohn-Sham
    solve per trial, loss, adjoint and gradient) of the 8^3-cell Q2
    two-electron workload from v_xc = 0, in this process.  The target density
    (oracle SCF) is set up outside the timing.  Returns (iterations, seconds)."""
    from oracle import fe, inverse, scf
    wl = W.cube8_q2_he()
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    d = scf.target_density(mesh, wl)
    op = inverse.Problem(mesh=mesh, v_fixed=d["v_fixed"], rho_data=d["rho_data"],
                         w=np.ones(mesh.L), n_electrons=wl.n_electrons, nstates=wl.nstates,
                         kT=wl.kT)
    st = inverse.State(v_xc=np.zeros(mesh.L))
    t0 = time.perf_counter()
    n = 0
    while n < max_iters:
        st = inverse.step(op, st)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return n, time.perf_counter() - t0


def oracle_iterations(threads: int, budget_s: float, max_iters: int):
    """_oracle_iterations_here in a child process whose BLAS / OpenMP pools are
    limited to `threads` (set before numpy loads).  Returns (iterations,
    seconds, threads)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    env["CUDA_VISIBLE_DEVICES"] = ""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-iterations",
                        str(budget_s), str(max_iters)], env=env, capture_output=True, text=True,
                       check=True)
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return out["iterations"], out["seconds"], threads


def oracle_hx_per_column(wl, budget_s: float = 6.0):
    """Seconds per column of the oracle's H~X (numpy FP64 cell loop) on the
    workload's full mesh, 2 columns at a time."""
    from oracle import fe
    mesh = fe.Mesh(wl.lo, wl.hi, wl.ncell, wl.order)
    ncol = 2
    X = W.random_block(mesh.L, ncol, wl.seed)
    v = np.zeros(mesh.L)
    t0 = time.perf_counter()
    reps = 0
    while True:
        mesh.apply_Htilde(v, X)
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 4:
            break
    return (time.perf_counter() - t0) / (reps * ncol)


def cpu_baseline(wl, budget_s: float = 8.0):
    """The oracle on the machine's host cores: full iterations of the small
    workload on one core and on all cores, and the oracle H~X of the bench
    workload's mesh; no extrapolation to the bench workload's iteration rate
    (an oracle iteration there takes hours, so it is not run)."""
    n1, s1, _ = oracle_iterations(1, budget_s, 10)
    cores = _cores()
    na, sa, _ = oracle_iterations(cores, budget_s, 10)
    hx_col = oracle_hx_per_column(wl) if wl.name != "cube8_q2_he" else None
    return {"value": na / sa, "unit": "iter/s", "cores": cores, "kind": "oracle",
            "sample": (f"full oracle iterations of cube8_q2_he (8^3 Q2 cells, 3,375 unknowns, "
                       f"2 electrons) from v_xc = 0: {na} in {sa:.2f} s on {cores} cores, "
                       f"{n1} in {s1:.2f} s on 1 core; the bench workload's oracle iteration "
                       "is not run (hours); its oracle H~X is timed per column"),
            "workload": "cube8_q2_he",
            "one_core": {"value": n1 / s1, "unit": "iter/s", "iterations": n1, "seconds": s1},
            "all_cores": {"value": na / sa, "unit": "iter/s", "iterations": na, "seconds": sa,
                          "cores": cores},
            "bench_workload_oracle_hx": (None if hx_col is None else
                                         {"workload": wl.name, "seconds_per_column": hx_col,
                                          "iteration": "not run"})}


def small_workload_gpu(device, steps=10, warmup=3):
    """GPU iterations/s of the mixed path on the cpu_baseline's small workload
    (the same config as the oracle's timed iterations)."""
    import torch
    wl = W.cube8_q2_he()
    pb, d = build_problem(wl, "mixed", device)
    v = torch.zeros(pb.L, dtype=torch.float64, device=device)
    for _ in range(warmup):
        pb.step(d["rho_data"], d["w"], v)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        pb.step(d["rho_data"], d["w"], v)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    pb.close()
    return {"workload": wl.name, "value": 1e3 / ms, "unit": "iter/s", "steps": steps,
            "warmup": warmup, "prec": "mixed"}


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


def fp64_arm(wl, d, device, steps, mixed_traj):
    """The plain FP64 GPU path on the same workload, from the same start, for
    `steps` steps (the first untimed); equal accuracy: e_L2 of both arms after
    every common step, and the two paths' gradients at the FP64 arm's last
    iterate."""
    import torch

    import paper_2510_10529_b300 as P
    pb = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                   kT=wl.kT, prec="fp64", cheb_degree=wl.cheb_degree, seed=wl.seed + 1,
                   device=device)
    pb.set_potential(d["v_fixed"], None)
    v = torch.zeros(pb.L, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream()
    traj, ms = [], []
    for k in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = pb.step(d["rho_data"], d["w"], v)
        e1.record(stream)
        torch.cuda.synchronize()
        traj.append(st["err_l2"])
        if k >= 1:
            ms.append(e0.elapsed_time(e1))
    common = min(len(traj), len(mixed_traj))
    rel = [abs(a - b) / b for a, b in zip(mixed_traj[:common], traj[:common])]
    pb.close()
    # both paths' gradients at the same potential (the FP64 arm's last
    # iterate), from fresh handles with the same fixed tight tolerances (the
    # adaptive ones depend on each handle's last e_L2)
    grads = {}
    for prec in ("fp64", "mixed"):
        q = P.Problem(wl.lo, wl.hi, wl.ncell, wl.order, wl.nstates, n_electrons=wl.n_electrons,
                      kT=wl.kT, prec=prec, cheb_degree=wl.cheb_degree, seed=wl.seed + 1,
                      eig_tol=1e-9, adj_tol=1e-10, device=device)
        q.set_potential(d["v_fixed"], v)
        _, g, _ = q.loss_grad(d["rho_data"], d["w"])
        grads[prec] = g
        q.close()
    grad_rel = ((grads["mixed"] - grads["fp64"]).norm() / grads["fp64"].norm()).item()
    out = {"value": (1e3 / statistics.mean(ms)) if ms else None, "unit": "iter/s",
           "steps_timed": len(ms), "untimed": 1, "ms_per_step": statistics.mean(ms) if ms else None,
           "err_l2": traj, "err_l2_mixed_same_steps": list(mixed_traj[:common]),
           "err_l2_rel_diff_max": max(rel) if rel else None,
           "grad_rel_diff_at_fp64_iterate": grad_rel,
           "grad_tolerances": {"eig_tol": 1e-9, "adj_tol": 1e-10}}
    return out


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
    traj = []
    for _ in range(args.warmup):
        traj.append(pb.step(rd, w, v_xc)["err_l2"])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    pb.profile_hx(True)
    launches0 = P.invdft_kernel_launches()
    stream = torch.cuda.current_stream()
    # timed steps: v_xc in from pinned host memory, the step, v_xc back out;
    # device time of the step alone (value) and wall time with the copies (e2e)
    v_host = v_xc.cpu().pin_memory()
    torch.cuda.synchronize()
    # INVDFT_PROFILE_TIMED=1 brackets the timed steps for a profiler started
    # with capture off (ncu --profile-from-start off); it changes no work
    profile_timed = os.environ.get("INVDFT_PROFILE_TIMED") == "1"
    if profile_timed:
        torch.cuda.profiler.start()
    dev_ms, wall_s, stats = 0.0, 0.0, []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        v_xc.copy_(v_host, non_blocking=True)
        e0.record(stream)
        st = pb.step(rd, w, v_xc)
        e1.record(stream)
        v_host.copy_(v_xc, non_blocking=True)
        torch.cuda.synchronize()
        wall_s += time.perf_counter() - t0
        dev_ms += e0.elapsed_time(e1)
        stats.append(st)
        traj.append(st["err_l2"])
    if profile_timed:
        torch.cuda.profiler.stop()
    launches = P.invdft_kernel_launches() - launches0
    prof = pb.profile_hx(False)
    defl = pb.profile_deflation()
    clk = clocks.stop()
    ms = dev_ms / args.steps
    ms_max = max_over_ranks(ms, world, device)
    e2e_s = max_over_ranks(wall_s / args.steps, world, device)
    value = whole_job_rate(1.0, world, ms_max / 1e3)
    e2e = {"value": whole_job_rate(1.0, world, e2e_s), "unit": "iter/s",
           "h2d_bytes_per_step": pb.L * 8, "d2h_bytes_per_step": pb.L * 8 + 8,
           "steps": "the timed steps (same as value)"}
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pk = peaks()
    peak_gbs = pk["hbm_gbs"] if pk else 6400.0
    ne, cells = (wl.order + 1) ** 3, wl.ncell ** 3

    def kind_summary(k, label):
        r = prof[k]
        nl = int(r["launches"])
        if nl == 0:
            return None
        cols = r["flops"] / (2.0 * ne * ne * cells) / nl     # columns per launch (exact)
        ach = r["bytes"] / (r["ms"] * 1e6)
        out = {"kernel": label, "launches": nl, "avg_launch_ms": r["ms"] / nl,
               "columns_per_launch": cols, "algorithmic_bytes_per_launch": r["bytes"] / nl,
               "achieved_gbs": ach, "hbm_frac": ach / peak_gbs,
               "ms_per_step": r["ms"] / args.steps}
        if k != "tf32" and abs(cols - round(cols)) < 1e-9:
            out["tuned_variant_seglen"] = {e: _schedule(vs) for e, vs in
                                           pb.hx_config(int(round(cols)), k == "fp64").items()}
        return out

    minres_kind = "fp32" if args.prec == "mixed" else "fp64"
    km = kind_summary(minres_kind, "hx_sweep_kernel: H~X of the MINRES iterations and the "
                      "other plain launches (" + ("FP32" if args.prec == "mixed" else "FP64")
                      + " sweep form, CUDA cores)")
    kf = kind_summary("fp32_filter", "hx_sweep_kernel: FP32 H~X of the defect-corrected "
                      "Chebyshev filter (W and E terms, CUDA cores)")
    kt = kind_summary("tf32", "hx_tc_kernel: TF32 H~X of the Chebyshev filter (tensor cores)")
    traffic = None
    if km and args.prec == "mixed" and HX_SWEEP_DRAM_BYTES_PER_NODE_COL:
        traffic = HX_SWEEP_DRAM_BYTES_PER_NODE_COL * pb.L * km["columns_per_launch"]
    roof = None
    if km:
        roof = {"bound": "hbm", "achieved": km["achieved_gbs"], "peak": peak_gbs, "unit": "GB/s",
                "frac": km["hbm_frac"], "traffic": traffic,
                "traffic_source": (f"ncu DRAM bytes per (node, column), {HX_SWEEP_DRAM_SOURCE}, "
                                   "scaled by unknowns x columns of the in-step launches"
                                   if traffic else "no capture of the current kernel"),
                "kernel": km["kernel"], "launches": km["launches"],
                "avg_launch_ms": km["avg_launch_ms"],
                "columns_per_launch": km["columns_per_launch"],
                "peak_source": "measured" if pk else "fallback",
                "algorithmic_bytes_per_launch": km["algorithmic_bytes_per_launch"]}
    def defl_summary(k, label):
        r = defl[k]
        nl = int(r["launches"])
        if nl == 0:
            return None
        ach = r["bytes"] / (r["ms"] * 1e6)
        return {"kernel": label, "launches": nl, "avg_launch_ms": r["ms"] / nl,
                "algorithmic_bytes_per_launch": r["bytes"] / nl, "achieved_gbs": ach,
                "hbm_frac": ach / peak_gbs, "ms_per_step": r["ms"] / args.steps}

    deflation = {"gram": defl_summary("gram", "defl_gram_tc_kernel: C = Psi^T Z of the MINRES "
                                      "deflation (tcgen05, split TF32)"),
                 "update": defl_summary("update", "defl_update_tc_kernel: Z -= Psi C with the "
                                        "fused column dot (tcgen05, split TF32)")}
    col_applies = sum(prof[k]["flops"] for k in prof) / (2.0 * ne * ne * cells)
    rates = measured_rates()
    hx = None if args.no_hx else hx_benchmark(device, rates=rates)
    fp64 = None
    if args.prec == "mixed" and args.fp64_steps > 0 and not args.ncell:
        pb.close()
        fp64 = fp64_arm(wl, d, device, args.fp64_steps, traj)
    small = None if args.no_cpu else small_workload_gpu(device)
    cpu = None
    if not args.no_cpu:
        try:
            cpu = cpu_baseline(wl)
        except Exception as exc:          # the GPU line must not be lost to a host failure
            cpu = {"value": None, "unit": "iter/s", "kind": "oracle", "error": repr(exc)}
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
        "clocks": clk, "hx": hx, "fp64_gpu": fp64, "small_workload_gpu": small,
        "measured_rates_tflops": rates,
        "hx_in_step": {"minres": km, "filter": kf, "filter_tf32": kt},
        "deflation_in_step": deflation,
        "step_stats": {"loss_last": stats[-1]["loss"], "err_l2_last": stats[-1]["err_l2"],
                       "err_l2": traj,
                       "cheb_passes": [s["cheb_passes"] for s in stats],
                       "minres_iters": [s["minres_iters_max"] for s in stats],
                       "ls_trials": [s["ls_trials"] for s in stats],
                       # host wall time of the forward solves (all line-search
                       # trials) and of the adjoint solve of each step
                       "t_forward_ms": [s["t_forward_ms"] for s in stats],
                       "t_adjoint_ms": [s["t_adjoint_ms"] for s in stats],
                       "col_applies_per_step": col_applies / args.steps,
                       "hx_ms_share": sum(prof[k]["ms"] for k in prof) / (ms_max * args.steps)},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
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
    """The oracle as it stands on the host cores: each step is one full oracle
    iteration of the 8^3-cell Q2 two-electron workload (all cores), after W
    untimed ones; the bench workload's oracle H~X per column is measured and
    reported beside it (its iteration is not run: hours)."""
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]()
    small = W.cube8_q2_he()
    cores = _cores()
    n_w, s_w, _ = oracle_iterations(cores, 1e9, args.warmup) if args.warmup else (0, 0.0, cores)
    n, sec, _ = oracle_iterations(cores, 1e9, args.steps)
    v = n / sec
    hx_col = oracle_hx_per_column(wl) if wl.name != small.name else None
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / n,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": small.name, "cells": f"{small.ncell}^3", "order": small.order,
                       "unknowns": small.n_interior, "nstates": small.nstates,
                       "n_electrons": small.n_electrons, "parallelism": "cpu",
                       "note": (f"the oracle iteration of {wl.name} takes hours and is not run; "
                                "this arm times full oracle iterations of the small workload "
                                "(the GPU arm reports its own rate on it as "
                                "small_workload_gpu)")},
            "cpu_baseline": {"value": v, "unit": "iter/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} full oracle iterations of {small.name} "
                                       f"(after {n_w} untimed), {sec:.2f} s, {cores} cores"},
            "bench_workload_oracle_hx": (None if hx_col is None else
                                         {"workload": wl.name, "seconds_per_column": hx_col,
                                          "iteration": "not run"}),
            "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_iterations:
        n, sec = _oracle_iterations_here(float(args.oracle_iterations[0]),
                                         int(args.oracle_iterations[1]))
        print(json.dumps({"iterations": n, "seconds": sec}))
        return
    if args.hx_case:
        n, k, kind = args.hx_case
        if kind not in ("tf32", "fp32", "fp64"):
            raise SystemExit("--hx-case KIND must be tf32, fp32 or fp64")
        hx_case(int(n), int(k), kind, "cuda", args.hx_variant, args.hx_seglen)
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
