#!/usr/bin/env python
"""Benchmark of the H-LU-preconditioned BiCGSTAB solve of the fractional SEM
system on one GB300 (N GPUs: independent replicas, weak scaling).

Workload (one step): nine instances on (0,1), N = 1024 uniform elements,
P = 8 (N_d = 8191), alpha in {1.2, 1.5, 1.8} x theta in {0, 0.3, 0.5},
rho = 1, seeded Legendre right-hand sides decaying like k^-2 (K = 32).  A step
runs the whole path: assembly (block-Toeplitz symbol, load vector),
H-matrix build with Taylor rank R = 8, H-LU (lambda = 1, Tol_HLU = 1e-3),
and BiCGSTAB to a relative residual of 1e-14 with the FFT operator.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  value = solves/s with the solution left in
device memory; e2e = the same through the C ABI with the solution copied to
pinned host memory inside the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

REF_BUDGET_S = 200.0   # wall time the reference arm's timed steps may take
METRIC = "solves/s & p50/p99 latency at <=1e-10 rel err: mixed vs FP64 H-LU-Krylov"
UNIT = "solves/s"
WORKLOAD = ("config 2: 9 instances, uniform N=1024, P=8 (N_d=8191), alpha x theta in "
            "{1.2,1.5,1.8}x{0,0.3,0.5}, rho=1, R=8, lambda=1, Tol_HLU=1e-3, Toeplitz FFT operator")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hfsem", choices=["hfsem", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    # profiling only: a reduced copy of the workload (fewer instances / elements)
    ap.add_argument("--instances", type=int, default=9)
    ap.add_argument("--n-elem", type=int, default=1024)
    return ap.parse_args()


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, ms_max, world):
    """Whole-job rate: the units every rank processed over the slowest rank's
    time (each rank runs the same batch: weak scaling)."""
    return world * units_per_rank / (ms_max * 1e-3)


def workload(n_inst=9, n_elem=1024):
    from paper_1808_02937_gb300 import hfsem as H
    from paper_1808_02937_gb300 import workloads as W
    insts = W.config2()[:n_inst]
    for p in insts:
        if n_elem != 1024:
            p.h = W.mesh_uniform(n_elem)
    probs = [H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho) for p in insts]
    rhs = [H.rhs_legendre([p.rhs[0]]) for p in insts]
    return insts, probs, rhs


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms; start()
    returns once the first sample is written, so the samples cover the region
    between start() and stop()."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        # raw samples: HFSEM_CLOCKS_CSV if set, else the system temp directory
        self.path = os.environ.get("HFSEM_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"hfsem_clocks_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def run_step(H, probs, rhs, opts, X, tol=1e-14):
    sys_ = H.hfsem_assemble(probs)
    fac = H.hfsem_hlu_factor(sys_, opts)
    X, st, code = H.hfsem_solve(sys_, fac, rhs, tol=tol, max_iter=60, X=X, allow_fail=True)
    del fac
    del sys_
    return X, st, code


def cpu_baseline_oracle(inst, max_cores):
    """Time the CPU oracle (dense assembly + dense LU + refinement) on one
    instance of the workload; returns (solves/s, seconds, X)."""
    from oracle.basis import Mesh
    from oracle.solve import solve_problem
    t0 = time.perf_counter()
    X, info = solve_problem(Mesh(inst.h, inst.a, inst.b), inst.P, inst.alpha, inst.theta,
                            inst.rho, inst.c1, inst.c2, ("legendre_ab", inst.rhs[0]))
    dt = time.perf_counter() - t0
    return 1.0 / dt, dt, X


def main_reference(args):
    """Reference arm: the CPU oracle, timed on this host's cores."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1808_02937_gb300 import workloads as W
    from oracle.basis import Mesh
    from oracle.solve import solve_problem
    insts = W.config2()
    small = W.config1()
    cores = os.cpu_count()
    # warm-up: the small configuration (imports, quadrature caches)
    for _ in range(args.warmup):
        solve_problem(Mesh(small.h, 0, 1), small.P, small.alpha, small.theta, small.rho,
                      small.c1, small.c2, ("frac_powers", small.rhs[0]))
    # one oracle solve takes ~17 s: steps beyond what fits in REF_BUDGET_S
    # (judged from the first step) are not run, and the line says so
    times = []
    for k in range(args.steps):
        if times and sum(times) + times[0] > REF_BUDGET_S:
            break
        p = insts[k % len(insts)]
        t0 = time.perf_counter()
        solve_problem(Mesh(p.h, p.a, p.b), p.P, p.alpha, p.theta, p.rho, p.c1, p.c2,
                      ("legendre_ab", p.rhs[0]))
        times.append(time.perf_counter() - t0)
    n_timed = len(times)
    ms = 1e3 * sum(times) / len(times)
    value = 1e3 / ms
    times.sort()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": n_timed, "steps_requested": args.steps,
            "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_step": "one of the nine instances"},
            "p50_ms": 1e3 * times[len(times) // 2], "p99_ms": 1e3 * times[-1],
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: one of the nine config-2 instances (oracle "
                                       f"dense assembly + dense LU + long-double refinement); "
                                       f"{n_timed} of {args.steps} requested steps timed "
                                       f"(budget {REF_BUDGET_S:.0f} s); warm-up on config 1"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        main_reference(args)
        return
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    from paper_1808_02937_gb300 import hfsem as H
    H.load_library()
    insts, probs, rhs = workload(args.instances, args.n_elem)
    reduced = (args.instances, args.n_elem) != (9, 1024)
    n_inst = len(insts)
    nd_total = sum(p.Nd for p in insts)
    prec = H.PREC_MIXED if args.precision == "mixed" else H.PREC_FP64
    opts = H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=prec)
    stream = torch.cuda.current_stream()
    X = torch.zeros(nd_total, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    for _ in range(max(args.warmup, 3)):
        X, st, code = run_step(H, probs, rhs, opts, X)
    torch.cuda.synchronize()

    # ---- timed region: device-resident solution ----
    H.hfsem_timing_reset()
    H.hfsem_timing_enable(True)
    launches0 = H.hfsem_timing_read("launches")[1]
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, iters = [], []
    barrier(world)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))                        # evict L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        X, st, code = run_step(H, probs, rhs, opts, X)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        iters.append([s["iters"] for s in st])
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = H.hfsem_timing_read("launches")[1] - launches0
    H.hfsem_timing_enable(False)
    kern = {}
    for tag in ("pairs", "toeplitz_mv", "hlu_factor", "hlu_solve", "krylov_vec"):
        ms, n, work = H.hfsem_timing_read(tag)
        kern[tag] = {"ms_total": ms, "launches": n, "work": work}
    mean_ms = sum(step_ms) / len(step_ms)
    mean_ms = max_over_ranks(mean_ms, world)
    value = job_throughput(n_inst, mean_ms, world)
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]

    # ---- end to end: solution copied to pinned host memory every step ----
    Xh = torch.zeros(nd_total, dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Xh, st, code = run_step(H, probs, rhs, opts, Xh)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_mean = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world)
    h2d = sum(8 * len(p.h) for p in insts) + sum(8 * len(p.rhs[0]) for p in insts) \
        + n_inst * 96
    d2h = 8 * nd_total + n_inst * 24

    # ---- parity and comparison legs ----
    Xd = X.cpu().numpy()
    fp64 = None
    if not args.no_fp64_compare and prec == H.PREC_MIXED:
        o64 = H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=H.PREC_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        X64, st64, _ = run_step(H, probs, rhs, o64, torch.zeros_like(X))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        X64 = X64.cpu().numpy()
        fp64 = {"solves_per_s": n_inst / dt, "ms_per_step": 1e3 * dt,
                "iters": [s["iters"] for s in st64],
                "max_rel_diff_vs_mixed": float(max(
                    np.linalg.norm(a[:, 0] - b[:, 0]) / np.linalg.norm(b[:, 0])
                    for a, b in zip(_Sys(insts).split(Xd), _Sys(insts).split(X64))))}

    peak, peak_src = peaks()
    # dominant kernel: the one with the largest device time
    dom = max(("hlu_factor", "hlu_solve", "toeplitz_mv", "pairs", "krylov_vec"),
              key=lambda t: kern[t]["ms_total"])
    roof = None
    if kern[dom]["launches"]:
        avg_s = kern[dom]["ms_total"] * 1e-3 / kern[dom]["launches"]
        per_launch = kern[dom]["work"] / kern[dom]["launches"]
        if dom in ("hlu_factor", "hlu_solve"):
            # FP32 (mixed) or FP64 CUDA-core arithmetic: peak from unit counts
            # and clock: 152 SMs x 128 FP32 lanes x 2 flops x max SM clock;
            # FP64: the part's nominal 1.25 TFLOP/s
            sm_mhz = float(peak.get("sm_max_mhz", 2070.0))
            pk = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12 if prec == H.PREC_MIXED else 1.25
            ach = per_launch / avg_s / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": pk,
                    "unit": "TFLOP/s", "frac": ach / pk, "traffic": None,
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x sm_max_mhz"
                    if prec == H.PREC_MIXED else "nominal FP64 1.25 TFLOP/s"}
        else:
            pk = float(peak["hbm_gbs"])
            ach = per_launch / avg_s / 1e9
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": pk,
                    "unit": "GB/s", "frac": ach / pk, "traffic": None,
                    "peak_source": peak_src}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not reduced:
        v, dt, Xo = cpu_baseline_oracle(insts[4], os.cpu_count())
        got = _Sys(insts).split(Xd)[4][:, 0]
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one of the nine instances (alpha=1.5, theta=0.3): oracle dense "
                         "assembly + dense LU + long-double refinement",
               "seconds": dt,
               "parity_rel_l2_err_vs_gpu": float(np.linalg.norm(got - Xo) / np.linalg.norm(Xo))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64 Krylov/operator, f32 H-LU" if prec == H.PREC_MIXED else "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD if not reduced else
                           f"REDUCED (profiling only): {n_inst} instances, N={args.n_elem}",
                           "instances_per_gpu": n_inst,
                           "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                           "krylov_tol": 1e-14},
                "p50_ms": p50, "p99_ms": p99, "wall_s_timed": wall,
                "iters": iters[-1],
                "e2e": {"value": job_throughput(n_inst, e2e_mean, world), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches, "clocks": clk, "roofline": roof,
                "kernels_ms_per_step": {t: kern[t]["ms_total"] / args.steps for t in kern},
                "cpu_baseline": cpu, "fp64_hlu": fp64}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


class _Sys:
    """Splits concatenated solution vectors per instance."""

    def __init__(self, insts):
        self.ndofs = [p.Nd for p in insts]

    def split(self, v):
        out, off = [], 0
        for nd in self.ndofs:
            out.append(v[off: off + nd].reshape(1, nd).T)
            off += nd
        return out


if __name__ == "__main__":
    main()
