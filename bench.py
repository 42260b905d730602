#!/usr/bin/env python3
"""Throughput of warm-started mixed-precision multigrid Poisson solves on one GB300.

Workload, one step: ten periodic Poisson solves A phi = delta_t on a 512^3 mesh,
delta_t = delta_0 + 0.05 t eta (t = 0..9; delta_0, eta seeded zero-mean
unit-variance Gaussian random fields with P(k) ~ k^-2).  t = 0 starts from
phi = 0, every later solve is warm-started from the previous phi (defect
correction, Sec. 3.2), each runs V(3,3) Chebyshev cycles in FP32 inside the
double-float outer refinement until ||F - A phi|| / ||F|| <= 1e-6.
Metric: solves/s (whole job, all ranks).  Inputs (1 GiB each) are larger than L2.

Also reported: per-kernel HBM roofline of the finest-level kernels (CUDA events
on the solver's stream during the timed region), the end-to-end rate through the
host-buffer C-ABI call, the plain FP64 V-cycle and cuFFT spectral solves of the
same sources on the same GPU, SM clocks sampled during the timed region, and the
CPU oracle timed on a bounded sample.

--impl reference times the CPU oracle (the reference implementation of this
build) on a bounded sample per step instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solves/s to rel. residual 1e-6 at 512^3 (warm-started sequence of 10 sources)"
UNIT = "solves/s"
# algorithmic bytes per finest-level cell of each timed kernel family
BYTES_PER_CELL = {
    "down0": 4 + 4 + 0.5,          # read r, write e, write R(r - A e) at 1/8 size
    "up0": 4 + 4 + 0.5 + 4,        # read e, r, coarse e at 1/8; write e
    "df0": 8 + 4 + 8 + 8 + 4,      # read phi (df), e, F (df); write phi (df), r
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=512)
    p.add_argument("--seq", type=int, default=10)
    p.add_argument("--tol", type=float, default=1e-6)
    p.add_argument("--degree", type=int, default=3)
    p.add_argument("--no-fused", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip e2e, baselines and CPU oracle legs")
    p.add_argument("--max-vcycles", type=int, default=40)
    p.add_argument("--only", choices=["moving_mesh", "differentiable", "batched", "fixed_2_cycles", "predictors",
                                      "pm_force", "e2e", "coarse_store"],
                   help="run one extra workload alone and print its JSON object (no headline line)")
    p.add_argument("--no-autotune", action="store_true", help="batched leg: default grid and tiles")
    p.add_argument("--print-source-digests", action="store_true",
                   help="print the source digest of each profiled kernel family and exit")
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "down0": ["legs.cuh", "legs.cu", "packed.cuh", "stencil.cuh", "common.cuh", "host_math.h"],
    "up0": ["legs.cuh", "legs.cu", "packed.cuh", "stencil.cuh", "common.cuh", "host_math.h"],
    "df0": ["dfk.cuh", "fused_kernels.cu", "packed.cuh", "stencil.cuh", "common.cuh", "host_math.h"],
}


def kernel_source_digest(family):
    """sha256 (first 16 hex digits) of the sources that define a kernel family."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[family]:
        with open(os.path.join(ROOT, "paper_2607_10983_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(family):
    """DRAM bytes per cell of a kernel family from the committed ncu summary table
    (profiles/ncu_traffic.txt), or None when the kernel's sources changed since."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        with open(path) as fh:
            for line in fh:
                cols = [c.strip() for c in line.strip().strip("|").split("|")]
                if len(cols) >= 5 and cols[0] == family:
                    if cols[4] != kernel_source_digest(family):
                        return None
                    return float(cols[3])
    except (OSError, ValueError, KeyError):
        return None
    return None


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [v.strip() for v in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
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


def aggregate(world, seq, steps, ms_local):
    """Whole-job rate: every rank's solves over the slowest rank's time (weak scaling)."""
    ms_total = max_over_ranks(ms_local, world)
    return ms_total, world * seq * steps / (ms_total / 1000.0)


def sources(n, seq, rank):
    """Host float64 sources of the warm-started sequence (seeds 2 and 3, shifted per rank)."""
    from synth import grf
    d0 = grf(n, 2 + 1000 * rank)
    eta = grf(n, 3 + 1000 * rank)
    return [d0 + (0.05 * t) * eta for t in range(seq)]


# ------------------------------------------------------------------ CPU oracle

def workload_config(args, levels):
    """The workload both arms run (the same dict on both lines)."""
    return {"workload": f"periodic 3-D Poisson {args.n}^3, warm-started sequence of {args.seq} GRF sources "
                        f"(P(k)~k^-2), tol {args.tol:g}, V({args.degree},{args.degree}) Chebyshev, {levels} levels",
            "n": args.n, "sources": args.seq, "tol": args.tol, "levels": levels,
            "l2": "inputs larger than L2 (1 GiB per field)"}


def oracle_sample(src0, src1, args):
    """The C FP64 V-cycle oracle (OpenMP over all host cores) on the first two solves of the
    sequence: t = 0 from zero, t = 1 warm-started from the oracle's own t = 0 solution."""
    import numpy as np

    from oracle import cmg
    s = cmg.Solver(src0.shape, degree=args.degree)
    phi = np.zeros(src0.shape)
    cycles = []
    t0 = time.perf_counter()
    for F in (src0, src1):
        phi, h = s.solve(F, phi, tol=args.tol, max_cycles=args.max_vcycles)
        cycles.append(len(h) - 1)
    dt = time.perf_counter() - t0
    s.close()
    return {"value": 2.0 / dt, "unit": UNIT, "cores": cmg.threads(), "kind": "oracle",
            "sample": (f"C FP64 V-cycle oracle on {cmg.threads()} host threads: solves t = 0 (cold, {cycles[0]} "
                       f"cycles) and t = 1 (warm, {cycles[1]} cycles) of the {args.n}^3 sequence, {dt:.1f} s")}


def run_reference(args):
    """The oracle arm: the C FP64 V-cycle oracle runs the same warm-started sequence on all
    host cores.  One step is one solve of the sequence to the tolerance (t = 0 from zero,
    each later source from the previous solution; the sequence restarts from zero after
    its last source); solves/s = timed steps / timed seconds."""
    import numpy as np

    from oracle import cmg
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from synth import grf
    n, seq, tol = args.n, args.seq, args.tol
    d0, eta = grf(n, 2), grf(n, 3)
    s = cmg.Solver(n, degree=args.degree)
    phi = np.zeros((n, n, n))
    timed_s, cycles = 0.0, []
    for k in range(args.warmup + args.steps):
        t = k % seq
        if t == 0:
            phi[:] = 0.0
        F = d0 + (0.05 * t) * eta          # input formation, outside the timed interval
        t0 = time.perf_counter()
        phi, h = s.solve(F, phi, tol=tol, max_cycles=args.max_vcycles)
        dt = time.perf_counter() - t0
        if h[-1] > tol:
            raise RuntimeError(f"oracle solve {t} did not reach {tol:g}")
        if k >= args.warmup:
            timed_s += dt
            cycles.append(len(h) - 1)
    levels = s.levels
    s.close()
    value = args.steps / timed_s
    first = args.warmup % seq
    cpu = {"value": value, "unit": UNIT, "cores": cmg.threads(), "kind": "oracle",
           "sample": (f"C FP64 V-cycle oracle on {cmg.threads()} host threads; each step one {n}^3 solve of the "
                      f"sequence (timed sources t = {first}, {(first + 1) % seq}, ... cycling through 0..{seq - 1}), "
                      f"{sum(cycles) / len(cycles):.2f} cycles per solve")}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * timed_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, levels), parallelism=f"replicas x{world}"),
        "precision": "FP64 V-cycle",
        "cycles_per_solve": sum(cycles) / len(cycles),
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import numpy as np
    import torch

    import paper_2607_10983_gb300 as gb
    from paper_2607_10983_gb300 import _build

    world, rank, local = dist_setup(args.gpus)
    _build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    n, seq = args.n, args.seq
    cells = n ** 3

    host_src = sources(n, seq, rank)
    F = [torch.from_numpy(a).to(dev) for a in host_src]
    phi = torch.zeros((n, n, n), dtype=torch.float64, device=dev)
    solver = gb.Solver(n, prec="mixed", degree=args.degree, fused=not args.no_fused)
    stream = torch.cuda.current_stream()
    cycles_log = []

    def step(record=False):
        phi.zero_()
        for t in range(seq):
            _, st = solver.solve(F[t], phi, tol=args.tol, max_vcycles=args.max_vcycles)
            if st.status != 0:
                raise RuntimeError(f"solve {t} failed: status {st.status}, rel_res {st.rel_res:.3e}")
            if record:
                cycles_log.append(st.cycles)

    for _ in range(args.warmup):
        step()
    families = ["down0", "up0", "df0"] if not args.no_fused else ["smooth0", "df0"]
    solver.profile_begin(families)
    launches0 = gb.launch_count()
    torch.cuda.synchronize()
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = gb.launch_count() - launches0
    ms_total, value = aggregate(world, seq, args.steps, ev0.elapsed_time(ev1))
    prof = {f: solver.profile_read(f) for f in families}
    solver.profile_end()
    ms_per_step = ms_total / args.steps

    hbm_peak, peak_kind = measured_peaks()
    kernels = {}
    for f, (cnt, kms) in prof.items():
        if cnt == 0:
            continue
        bpc = BYTES_PER_CELL.get(f, 20.0 if f == "smooth0" else 0.0)
        avg_ms = kms / cnt
        gbs = bpc * cells / (avg_ms / 1000.0) / 1e9
        kernels[f] = {"launches": cnt, "avg_ms": avg_ms, "share_of_step": kms / ms_total,
                      "bytes_per_cell": bpc, "achieved_gbs": gbs, "frac": gbs / hbm_peak}
    dom = max(kernels, key=lambda f: kernels[f]["avg_ms"] * kernels[f]["launches"])
    tr = ncu_traffic(dom)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": kernels[dom]["achieved_gbs"], "peak": hbm_peak,
                "peak_kind": f"{peak_kind} copy bandwidth (burst)", "unit": "GB/s",
                "frac": kernels[dom]["achieved_gbs"] / hbm_peak,
                "traffic": (tr * cells if tr is not None else None)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(args, solver.levels), parallelism=f"replicas x{world}"),
        "precision": "FP32 V-cycle inside double-float defect correction" + ("" if not args.no_fused else ", unfused"),
        "cycles_per_solve": sum(cycles_log) / max(1, len(cycles_log)),
        "gpu_launches": launches,
        "roofline": roofline,
        "kernels": kernels,
    }
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks

    if not args.no_extras and rank == 0:
        line["e2e"] = e2e_leg(args, solver, host_src)
        line["baselines"] = baseline_legs(args, F, dev)
        line["fixed_2_cycles"] = fixed_cycles_leg(args, solver, F)
        line["coarse_store"] = coarse_store_leg(args, F, dev)
        line["predictors"] = predictors_leg(args, solver, F)
        line["krylov_2"] = krylov_leg(args, F)
        del F
        del phi
        solver.close()
        torch.cuda.empty_cache()
        line["differentiable_256"] = differentiable_leg(args, dev)
        line["moving_mesh_256"] = moving_mesh_leg(args, dev)
        line["pm_force_256"] = pm_force_leg(args, dev)
        torch.cuda.empty_cache()
        line["batched_48"] = batched_leg(args)
        line["cpu_baseline"] = oracle_sample(host_src[0], host_src[1], args)
    if rank == 0:
        print(json.dumps(line))
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def e2e_leg(args, solver, host_src):
    """Same sequence through mg_solve_host_sequence: pinned host sources in, pinned host
    solutions out, copies inside the timed region (overlapped with the neighbouring solves)."""
    import torch
    n, seq = args.n, args.seq
    pinned = [torch.from_numpy(a).pin_memory() for a in host_src]
    outs = [torch.empty((n, n, n), dtype=torch.float64).pin_memory() for _ in range(seq)]

    def step():
        sts = solver.solve_host_sequence(pinned, outs, tol=args.tol, max_vcycles=args.max_vcycles)
        if any(st.status != 0 for st in sts):
            raise RuntimeError("e2e sequence did not converge")

    step()
    steps = max(1, min(args.steps, 3))
    per_step = []
    for _ in range(steps):
        t0 = time.perf_counter()
        step()
        per_step.append(time.perf_counter() - t0)
    dt = sum(per_step)
    b = n ** 3 * 8
    return {"value": seq * steps / dt, "unit": UNIT, "h2d_bytes_per_step": seq * b,
            "d2h_bytes_per_step": seq * b, "ms_per_step": [1000.0 * x for x in per_step],
            "api": "mg_solve_host_sequence (pinned host buffers; the first solve starts from zero, each later one "
                   "from the previous solution on the device)"}


def baseline_legs(args, F, dev):
    """Plain FP64 V-cycle (one kernel per operation) and cuFFT spectral solves of the same sources."""
    import math

    import torch

    import paper_2607_10983_gb300 as gb
    n = args.n
    out = {}
    # plain FP64 V-cycle (one kernel per operation) on the headline's workload: the whole
    # sequence, t = 0 from zero and every later source warm-started from the previous phi
    s64 = gb.Solver(n, prec="fp64", degree=args.degree)
    phi = torch.zeros_like(F[0])
    s64.solve(F[1], phi.clone(), tol=1e-2, max_vcycles=1)
    cycles = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for f in F:
        _, st = s64.solve(f, phi, tol=args.tol, max_vcycles=args.max_vcycles)
        cycles.append(st.cycles)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out["plain_fp64_vcycle"] = {"solves_per_s": len(F) / dt, "cycles_per_solve": sum(cycles) / len(F),
                                "ms_per_cycle": 1000 * dt / sum(cycles), "cycles": cycles,
                                "sources": f"the headline sequence, t = 0..{len(F) - 1}, warm-started"}
    s64.close()
    del phi
    # cuFFT spectral solve of the same 7-point operator (torch.fft), FP64 and FP32
    kz = 2 * math.pi * torch.fft.fftfreq(n, device=dev, dtype=torch.float64)
    kx = 2 * math.pi * torch.fft.rfftfreq(n, device=dev, dtype=torch.float64)
    lam = -4.0 * (torch.sin(kz / 2)[:, None, None] ** 2 + torch.sin(kz / 2)[None, :, None] ** 2
                  + torch.sin(kx / 2)[None, None, :] ** 2)
    lam[0, 0, 0] = 1.0
    inv = 1.0 / lam
    inv[0, 0, 0] = 0.0
    for name, dt_ in (("cufft_fp64", torch.float64), ("cufft_fp32", torch.float32)):
        iv = inv.to(dt_)
        srcs = [f.to(dt_) for f in F]

        def solve(f):
            return torch.fft.irfftn(torch.fft.rfftn(f) * iv, s=(n, n, n))

        solve(srcs[0])
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        for f in srcs:
            solve(f)
        ev1.record()
        torch.cuda.synchronize()
        out[name] = {"solves_per_s": len(srcs) / (ev0.elapsed_time(ev1) / 1000.0),
                     "note": "rfftn, divide by the 7-point symbol, irfftn; the headline's 10 sources, resident"}
        sol = solve(srcs[0]).double()
        if name == "cufft_fp64":
            ref64 = sol
        else:
            out[name]["rel_l2_vs_fp64"] = float(torch.linalg.vector_norm(sol - ref64)
                                                / torch.linalg.vector_norm(ref64))
        del srcs, sol
    return out


def coarse_store_leg(args, F, dev):
    """The sequence with the corrections of levels below 128^3 stored in FP32 (the headline),
    BF16 or FP16 (opts.coarse_store): solves/s, cycles per solve and the last solution's
    relative L2 error against the FP64 cuFFT solve of the same operator."""
    import math

    import torch

    import paper_2607_10983_gb300 as gb
    n = args.n
    kz = 2 * math.pi * torch.fft.fftfreq(n, device=dev, dtype=torch.float64)
    kx = 2 * math.pi * torch.fft.rfftfreq(n, device=dev, dtype=torch.float64)
    lam = -4.0 * (torch.sin(kz / 2)[:, None, None] ** 2 + torch.sin(kz / 2)[None, :, None] ** 2
                  + torch.sin(kx / 2)[None, None, :] ** 2)
    lam[0, 0, 0] = 1.0
    Fk = torch.fft.rfftn(F[-1]) / lam
    Fk[0, 0, 0] = 0.0
    ref = torch.fft.irfftn(Fk, s=(n, n, n))
    del Fk, lam
    out = {}
    for store in ("fp32", "bf16", "fp16"):
        s = gb.Solver(n, prec="mixed", degree=args.degree, coarse_store=store)
        phi = torch.zeros_like(F[0])
        s.solve(F[1], phi.clone(), tol=1e-2, max_vcycles=1)
        cycles = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in F:
            _, st = s.solve(f, phi, tol=args.tol, max_vcycles=args.max_vcycles)
            cycles.append(st.cycles)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        err = float(torch.linalg.vector_norm(phi - ref) / torch.linalg.vector_norm(ref))
        out[store] = {"solves_per_s": len(F) / dt, "cycles_per_solve": sum(cycles) / len(F), "cycles": cycles,
                      "rel_l2_vs_fp64_fft": err}
        s.close()
        del phi
    out["note"] = ("corrections of levels below 128^3 rounded to the format before prolongation (the bottom "
                   "cycle's levels, 16^3 and below, stay FP32 inside it); timing includes the rounding passes")
    return out


def fixed_cycles_leg(args, solver, F):
    """The sequence at the paper's warm-start operating point: t = 0 solved to tol, each later
    source warm-started from the previous phi with at most 2 V-cycles (residual reported)."""
    import torch
    phi = torch.zeros_like(F[0])
    solver.solve(F[0], phi, tol=args.tol, max_vcycles=args.max_vcycles)
    phi.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rel = []
    for t in range(len(F)):
        _, st = solver.solve(F[t], phi, tol=args.tol, max_vcycles=args.max_vcycles if t == 0 else 2)
        rel.append(st.rel_res)
    dt = time.perf_counter() - t0
    return {"solves_per_s": len(F) / dt, "rel_res_per_source": rel,
            "note": "t = 0 to the tolerance, t >= 1 at most 2 V-cycles (status NOT_CONVERGED allowed)"}


def predictors_leg(args, solver, F):
    """The sequence with the warm-start predictors of Sec. 3.2: recycling (the headline
    path), linear and quadratic extrapolation over the previous solutions (mg_predict,
    one extra FP64 pass per solve, counted in the time).  Early steps use the highest
    order their history allows.  The synthetic sources drift exactly linearly in t, so
    extrapolation is near exact here; real PM sources are not."""
    import torch
    n, seq = args.n, len(F)
    ring = [torch.zeros((n, n, n), dtype=torch.float64, device=F[0].device) for _ in range(4)]
    out = {}
    for name, order in (("recycle", 0), ("linear", 1), ("quadratic", 2)):
        for b in ring:
            b.zero_()
        hist = []          # indices into ring, most recent first
        cycles = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(seq):
            if not hist or order == 0:
                cur = hist[0] if hist else 0          # cold start, or recycling in place
            else:
                cur = next(i for i in range(4) if i not in hist[:3])
                k = min(order, len(hist) - 1)
                solver.predict([ring[i] for i in hist[:k + 1]], order=k, out=ring[cur])
            _, st = solver.solve(F[t], ring[cur], tol=args.tol, max_vcycles=args.max_vcycles)
            cycles.append(st.cycles)
            hist = [cur] + [i for i in hist if i != cur]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"solves_per_s": seq / dt, "cycles_per_solve": sum(cycles) / seq, "cycles": cycles}
    del ring
    out["note"] = ("sources drift exactly linearly in t (delta_t = delta_0 + 0.05 t eta), so extrapolation "
                   "is near exact on this workload; the headline value uses recycling")
    return out


def pm_force_leg(args, dev):
    """Static PM force evaluation at 256^3: 256^3 particles (displaced lattice) on a 256^3
    mesh; CIC paint, solve, fourth-order gradient, read (the unit of the paper's
    force-evaluation cost tables).  Variants: cold solve to 1e-6, and warm starts from the
    previous step's potential (particles displaced 2% less) with at most 1 or 2 V-cycles
    (the paper's operating points).  Per-stage device times."""
    import torch

    import paper_2607_10983_gb300 as gb
    from synth import lattice_particles
    n = 256
    p_prev = torch.from_numpy(lattice_particles(n, n, 9, rms_displacement=1.96)).to(dev)
    p = torch.from_numpy(lattice_particles(n, n, 9, rms_displacement=2.0)).to(dev)
    s = gb.Solver(n)
    rho = s.cic_paint(p_prev, 1.0)
    phi_prev, _ = s.solve(rho, tol=args.tol, max_vcycles=args.max_vcycles)
    phi = torch.empty_like(phi_prev)
    force = torch.empty((p.shape[0], 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def step(warm, tol, maxv):
        if warm:
            phi.copy_(phi_prev)
        else:
            phi.zero_()
        ev[0].record(stream)
        s.cic_paint(p, 1.0, out=rho)
        ev[1].record(stream)
        _, st = s.solve(rho, phi, tol=tol, max_vcycles=maxv)
        ev[2].record(stream)
        ev[3].record(stream)
        s.force(phi, p, out=force)
        ev[4].record(stream)
        torch.cuda.synchronize()
        return st, [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]

    out = {}
    for name, warm, tol, maxv in (("cold_to_1e-6", False, args.tol, args.max_vcycles), ("warm_1_cycle", True, 0.0, 1),
                                  ("warm_2_cycles", True, 0.0, 2)):
        step(warm, tol, maxv)                    # warm-up
        reps, tot, stages = 3, 0.0, [0.0] * 4
        for _ in range(reps):
            st, t = step(warm, tol, maxv)
            tot += sum(t)
            stages = [a + b for a, b in zip(stages, t)]
        out[name] = {"ms": tot / reps, "cycles": st.cycles, "rel_res": st.rel_res,
                     "paint_solve_force_ms": [stages[0] / reps, stages[1] / reps, (stages[2] + stages[3]) / reps]}
    s.close()
    out["workload"] = ("256^3 particles (lattice + Zel'dovich-like displacement, rms 2 cells, seed 9) on a 256^3 "
                       "mesh; force = -grad4 phi read at the particles; context: the paper quotes 17.9 ms (FFT) "
                       "and 16.5 ms (warm MG, 1 cycle) per full PM step at 256^3 on one A100")
    return out


def krylov_leg(args, F):
    """The sequence with V-cycle-preconditioned CG corrections (Sec. 3.2; 2 CG steps, i.e.
    2 V-cycles, per defect-correction step), warm-started by recycling."""
    import torch

    import paper_2607_10983_gb300 as gb
    n = args.n
    s = gb.Solver(n, prec="mixed", degree=args.degree, krylov=2)
    phi = torch.zeros_like(F[0])
    s.solve(F[0], phi.clone(), tol=1e-2, max_vcycles=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps = []
    for f in F:
        _, st = s.solve(f, phi, tol=args.tol, max_vcycles=args.max_vcycles)
        steps.append(st.cycles)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return {"solves_per_s": len(F) / dt, "outer_steps_per_solve": sum(steps) / len(F),
            "vcycles_per_solve": 2 * sum(steps) / len(F)}


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, 1000.0 * (time.perf_counter() - t0)


def differentiable_leg(args, dev):
    """256^3 differentiable flat solve: loss = sum(w . grad4 phi), phi = solve(F) (mixed, to 1e-6);
    backward = adjoint solve.  Forward and backward wall times, and the gradient against central
    differences of the same GPU loss (solves to 1e-10) in 4 seeded source directions."""
    import numpy as np
    import torch

    import paper_2607_10983_gb300 as gb
    from synth import grf, vector_noise
    n = 256
    F = torch.from_numpy(grf(n, 4)).to(dev)
    w = torch.from_numpy(vector_noise(n, 5)).to(dev, torch.float32)
    s = gb.Solver(n)

    def fwd():
        Fd = F.clone().requires_grad_(True)
        return Fd, gb.GradDotLoss.apply(gb.MGSolve.apply(Fd, s, args.tol, args.max_vcycles), w, s, 4)

    fwd()[1].backward()                      # warm-up
    (Fd, loss), t_fwd = _timed(fwd)
    _, t_bwd = _timed(loss.backward)
    g = Fd.grad

    def L(FF):
        ph, _ = s.solve(FF, tol=1e-10, max_vcycles=60)
        return float(s.grad_dot(ph, w, 4))

    Fd2 = F.clone().requires_grad_(True)
    gb.GradDotLoss.apply(gb.MGSolve.apply(Fd2, s, 1e-10, 60), w, s, 4).backward()
    worst = 0.0
    for seed in range(100, 104):
        v = torch.from_numpy(np.random.default_rng(seed).standard_normal((n, n, n))).to(dev)
        fd = (L(F + 1e-3 * v) - L(F - 1e-3 * v)) / 2e-3
        worst = max(worst, abs(fd - float((Fd2.grad * v).sum())) / max(1.0, abs(fd)))
    s.close()
    del g
    return {"forward_ms": t_fwd, "backward_ms": t_bwd, "fd_max_rel_diff": worst,
            "workload": "256^3 flat, F seed 4, w seed 5 (FP32), tol 1e-6 timed; FD eps 1e-3, directions seeds 100..103"}


def moving_mesh_leg(args, dev):
    """256^3 moving-mesh solve (19-point curvilinear operator of psi, FP32 coefficients,
    double-float refinement to 1e-6) and its adjoint (delta_bar, psi_bar): wall times, cycles,
    the finest-level Jacobi sweep's device time and GB/s, and central differences of the
    GPU loss sum(w . grad2 phi) in one delta and one psi direction."""
    import numpy as np
    import torch

    import paper_2607_10983_gb300 as gb
    from synth import grf, smoothed_grf, vector_noise
    n = 256
    psi = torch.from_numpy(smoothed_grf(n, 6, 4.0, 0.5)).to(dev)
    delta = torch.from_numpy(grf(n, 7)).to(dev)
    w = torch.from_numpy(vector_noise(n, 8).astype(np.float64)).to(dev)
    s = gb.Solver(n, op="curv")
    pbar = s.grad_T(w.to(torch.float32), 2)
    # warm-up of both solves (one-time scratch and the cycles' CUDA graphs), the timed
    # solves, then a solve with the sweep and the double-float residual timed per launch
    phi_w, _ = s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi)
    s.solve_adjoint(pbar, phi=phi_w, source=delta, want_psi_bar=True, tol=args.tol, max_vcycles=100)
    (phi, st), t_fwd = _timed(lambda: s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi))
    (res_adj), t_adj = _timed(lambda: s.solve_adjoint(pbar, phi=phi, source=delta, want_psi_bar=True,
                                                      tol=args.tol, max_vcycles=100))
    s.profile_begin(["curv0", "df0"])
    s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi)
    prof = {f: s.profile_read(f) for f in ("curv0", "df0")}
    s.profile_end()
    _, _, st_adj = res_adj
    hbm_peak, _ = measured_peaks()
    cells = n ** 3
    kern = {}
    for f, bpc in (("curv0", 40.0), ("df0", 48.0)):
        cnt, kms = prof[f]
        if cnt:
            gbs = bpc * cells / (kms / cnt / 1000.0) / 1e9
            kern[f] = {"launches": cnt, "avg_ms": kms / cnt, "bytes_per_cell": bpc, "achieved_gbs": gbs,
                       "frac": gbs / hbm_peak}
    # gradient check at 1e-10
    phi_t, _ = s.solve(delta, tol=1e-10, max_vcycles=200, psi=psi)
    dbar, psibar, _ = s.solve_adjoint(pbar, phi=phi_t, source=delta, want_psi_bar=True, tol=1e-10, max_vcycles=200)

    def L(d, p):
        ph, _ = s.solve(d, tol=1e-10, max_vcycles=200, psi=p)
        return float((w * s.grad(ph, 2)).sum())

    v = torch.from_numpy(np.random.default_rng(300).standard_normal((n, n, n))).to(dev)
    fd = (L(delta + 1e-3 * v, psi) - L(delta - 1e-3 * v, psi)) / 2e-3
    d_rel = abs(fd - float((dbar * v).sum())) / max(1.0, abs(fd))
    dp = torch.from_numpy(smoothed_grf(n, 400, 4.0, 0.5)).to(dev)
    fd = (L(delta, psi + 1e-2 * dp) - L(delta, psi - 1e-2 * dp)) / 2e-2
    p_rel = abs(fd - float((psibar * dp).sum())) / max(1.0, abs(fd))
    s.close()
    # the symmetric discretisation variant on the same workload (forward and adjoint)
    s = gb.Solver(n, op="curv", curv_sym=True)
    phi_w, _ = s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi)        # warm-up
    s.solve_adjoint(pbar, phi=phi_w, source=delta, want_psi_bar=True, tol=args.tol, max_vcycles=100)
    (phi_s, st_s), t_fwd_s = _timed(lambda: s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi))
    (res_s), t_adj_s = _timed(lambda: s.solve_adjoint(pbar, phi=phi_s, source=delta, want_psi_bar=True,
                                                      tol=args.tol, max_vcycles=100))
    s.profile_begin(["curv0"])
    s.solve(delta, tol=args.tol, max_vcycles=100, psi=psi)
    cnt, kms = s.profile_read("curv0")
    s.profile_end()
    gbs = 40.0 * cells / (kms / cnt / 1000.0) / 1e9
    sym = {"forward_ms": t_fwd_s, "forward_cycles": st_s.cycles, "forward_rel_res": st_s.rel_res,
           "adjoint_ms": t_adj_s, "adjoint_cycles": res_s[2].cycles,
           "curv0": {"launches": cnt, "avg_ms": kms / cnt, "bytes_per_cell": 40.0, "achieved_gbs": gbs,
                     "frac": gbs / hbm_peak},
           "rel_l2_vs_paper_scheme": float(torch.linalg.norm(phi_s - phi) / torch.linalg.norm(phi))}
    s.close()
    return {"forward_ms": t_fwd, "forward_cycles": st.cycles, "forward_rel_res": st.rel_res,
            "adjoint_ms": t_adj, "adjoint_cycles": st_adj.cycles, "kernels": kern,
            "fd_rel_diff": {"delta": d_rel, "psi": p_rel}, "symmetric_variant": sym,
            "workload": "256^3, psi seed 6 (Gaussian-smoothed GRF, sigma 4, Gershgorin |Hess psi| 0.5), "
                        "delta seed 7, w seed 8; V(2,2) Jacobi, tol 1e-6 timed; FD eps 1e-3 (delta), 1e-2 (psi)"}


def batched_leg(args):
    """48 independent cold solves, 16 each at 64^3, 96^3 and 128^3 (seeds 1000..1047), tol 1e-6:
    one persistent launch for all vs the same solves one at a time."""
    import numpy as np
    import torch

    import paper_2607_10983_gb300 as gb
    from synth import grf
    shapes = [(64,) * 3] * 16 + [(96,) * 3] * 16 + [(128,) * 3] * 16
    F = [torch.from_numpy(grf(s, 1000 + i)).cuda() for i, s in enumerate(shapes)]
    phis = [torch.zeros_like(f) for f in F]
    batch = gb.Batch(shapes, degree=args.degree)
    if args.no_autotune:   # default grid (one CTA per SM) and tiles: fixed launches for profiling
        blocks, tiles = "default", batch.tiles()
    else:
        blocks, tiles = batch.autotune(F, phis, tol=args.tol, max_vcycles=args.max_vcycles)
    batch.use_graph(True)
    for p in phis:
        p.zero_()
    batch.solve(F, phis, tol=args.tol, max_vcycles=args.max_vcycles)   # captures the graph
    reps = 3
    lat, total = [], 0.0
    for _ in range(reps):
        for p in phis:
            p.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        stats, times = batch.solve(F, phis, tol=args.tol, max_vcycles=args.max_vcycles)
        total += time.perf_counter() - t0
        lat += times
        if any(st.status != 0 for st in stats):
            raise RuntimeError("batched solve did not converge")
    out = {"batched": {"solves_per_s": len(shapes) * reps / total, "p50_ms": float(np.percentile(lat, 50)),
                       "p99_ms": float(np.percentile(lat, 99)), "blocks": blocks, "tiles": tiles, "cuda_graph": True,
                       "cycles_per_solve": float(np.mean([st.cycles for st in stats]))}}
    batch.close()
    solvers = {s: gb.Solver(s, degree=args.degree) for s in set(shapes)}
    seq_lat = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for f, s in zip(F, shapes):          # warm-up
        solvers[s].solve(f, torch.zeros_like(f), tol=args.tol, max_vcycles=args.max_vcycles)
    t0 = time.perf_counter()
    for _ in range(reps):
        for f, s in zip(F, shapes):
            ph = torch.zeros_like(f)
            ev0.record()
            solvers[s].solve(f, ph, tol=args.tol, max_vcycles=args.max_vcycles)
            ev1.record()
            ev1.synchronize()
            seq_lat.append(ev0.elapsed_time(ev1))
    dt = time.perf_counter() - t0
    out["one_at_a_time"] = {"solves_per_s": len(shapes) * reps / dt, "p50_ms": float(np.percentile(seq_lat, 50)),
                            "p99_ms": float(np.percentile(seq_lat, 99))}
    out["workload"] = "48 cold solves to 1e-6: 16 x 64^3, 16 x 96^3, 16 x 128^3, GRF P(k)~k^-2, seeds 1000..1047"
    for s in solvers.values():
        s.close()
    return out


def run_only(args):
    import torch

    from paper_2607_10983_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.only == "moving_mesh":
        out = moving_mesh_leg(args, dev)
    elif args.only == "differentiable":
        out = differentiable_leg(args, dev)
    elif args.only == "batched":
        out = batched_leg(args)
    elif args.only == "pm_force":
        out = pm_force_leg(args, dev)
    else:
        import paper_2607_10983_gb300 as gb
        host = sources(args.n, args.seq, 0)
        F = [torch.from_numpy(a).to(dev) for a in host]
        solver = gb.Solver(args.n, prec="mixed", degree=args.degree, fused=not args.no_fused)
        if args.only == "e2e":
            out = e2e_leg(args, solver, host)
        elif args.only == "coarse_store":
            out = coarse_store_leg(args, F, dev)
        else:
            leg = fixed_cycles_leg if args.only == "fixed_2_cycles" else predictors_leg
            out = leg(args, solver, F)
        solver.close()
    print(json.dumps({args.only: out}))


def main():
    args = parse()
    if args.print_source_digests:
        for f in KERNEL_SOURCES:
            print(f, kernel_source_digest(f))
        return
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
