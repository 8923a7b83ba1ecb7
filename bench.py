#!/usr/bin/env python
"""Benchmark of the immersed-boundary DVM step on GB300.

Metric: DVM cell x velocity updates per second (fluid cells x discrete
velocities advanced per step, summed over ranks), with the achieved fraction
of the HBM roofline of the dominant kernel (the transport/relaxation sweep).

Default workload: the 3D sphere, 96^3 cells on [-4,4]^3, 20^3 velocities on
[-5,5]^3, Kn 0.1, Ma 0.5, mixed precision (FP32 f, FP64 wall balance, forces
and residual): the largest configuration that fits one GPU (7.08G cell x
velocity pairs, 58 GB of state).  The 2D cylinder (512^2 cells on [-8,8]^2,
48^2 velocities on [-6,6]^2, Kn 0.1, Ma 0.5, mixed) is measured in the same
run and reported under the key "cylinder_512".  A step is the whole hot path:
ghost band (upwind-weighted interpolation, wall density, cut-cell blend, ghost
values), surface forces, transport and relaxation of every fluid cell,
moments and residual.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 the script runs under torch.distributed.run: every rank advances
its own replica of the case (the method has no exchange between independent
cases), timing is the max over ranks, and the value is the sum over ranks.
"--impl reference" times the CPU oracle on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "cylinder_512": lambda p, kn=0.1: __import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).cylinder_512(
        kn, p),
    "sphere_96": lambda p: __import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).sphere_96(p),
    "cylinder_48": lambda p: dict(__import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).cylinder_48(),
                                  precision=p),
    "cavity_64": lambda p: __import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).cavity(
        n=64, nv=100, precision=p),
    "sphere_96_stretched": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                                fromlist=["x"]).sphere_96_stretched(p),
    "sphere_supersonic": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                              fromlist=["x"]).sphere_supersonic(precision=p),
    "naca_supersonic": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                            fromlist=["x"]).naca_supersonic(precision=p),
    "cylinder_hypersonic": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                                fromlist=["x"]).cylinder_hypersonic(precision=p),
    "tree_2d": lambda p: __import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).tree_2d(precision=p),
    "cylinder_hypersonic_tree": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                                     fromlist=["x"]).cylinder_hypersonic_tree(precision=p),
    "naca_supersonic_tree": lambda p: __import__("paper_2512_20252_gb300.workloads",
                                                 fromlist=["x"]).naca_supersonic_tree(precision=p),
    "sphere_96_tree": lambda p: __import__("paper_2512_20252_gb300.workloads", fromlist=["x"]).sphere_96_tree(precision=p),
    "batched_2d": None,  # a list of cases: see bench_batch
    "served": None,      # a request stream: see bench_serve
}
DESCRIPTIONS = {
    "cylinder_512": "2D cylinder r=0.5, 512x512 cells on [-8,8]^2, 48x48 trapezoid velocities on [-6,6]^2, Kn=0.1, Ma=0.5",
    "sphere_96": "3D sphere r=0.5, 96^3 cells on [-4,4]^3, 20^3 trapezoid velocities on [-5,5]^3, Kn=0.1, Ma=0.5",
    "cylinder_48": "2D cylinder r=0.5, 48x48 cells on [-4,4]^2, 24x24 trapezoid velocities on [-5,5]^2, Kn=0.1, Ma=0.3",
    "cylinder_hypersonic": "2D cylinder r=1, 1536x1536 cells on [-16,16]^2, 60x60 trapezoid velocities on "
                           "[-10,10]^2, Kn=0.1, Ma=5, T_w=1, nonnegative ghost values",
    "naca_supersonic": "2D NACA0012 airfoil (chord 1, AoA 0, T_w=1), Ma=2, Kn=0.026, 1000x1400 cells on "
                       "[-3,7]x[-7,7], 60x60 trapezoid velocities on [-4,8]x[-6,6]",
    "sphere_supersonic": "3D sphere r=0.5, 64^3 cells on [-4,4]^3, Ma=3.834, Kn=0.03, T_w=5.90, 24^3 stretched "
                         "velocities on [-7.29,7.29]^3 (central spacing 0.2275), nonnegative ghost values",
    "sphere_96_stretched": "3D sphere r=0.5, 96^3 cells on [-4,4]^3, 20^3 stretched velocities on [-5,5]^3 "
                           "(central spacing 0.25), Kn=0.1, Ma=0.5",
    "cavity_64": "2D lid-driven cavity [0,1]^2 with a cylinder of diameter 0.25 at its centre, 64x64 cells, "
                 "100x100 trapezoid velocities on [-5,5]^2, diffuse walls at T_w=1, lid 0.15, Kn=0.075",
    "tree_2d": "2D tree-refined grid: a 128x128 root on [-8,8]^2 refined around the origin to level 1 within 4, "
               "2 within 2 and 3 within 1 (finest edge 1/64), 2:1 balanced, 45,436 leaves in Z order, 48x48 "
               "trapezoid velocities on [-6,6]^2, Kn=0.1, Ma=0.5, no body, a 20% density bump over the refined "
               "region at the start",
    "cylinder_hypersonic_tree": "2D cylinder r=1 at Ma 5, Kn 0.1 on a tree: a 128x128 root on [-16,16]^2 refined "
                                "about the centre to level 1 within 8, 2 within 4, 3 within 2.2, 4 within 1.5 "
                                "(finest edge 1/64 at the wall), 2:1 balanced, 69,148 leaves in Z order, 60x60 "
                                "trapezoid velocities on [-10,10]^2, T_w=1, nonnegative ghost values",
    "naca_supersonic_tree": "NACA0012 (chord 1, 400-vertex polygon) at Ma 2, Kn 0.026, AoA 0 on a tree: an 80x112 "
                            "root on [-3,7]x[-7,7] refined about the chord to level 1 within 1.5, 2 within 0.6, 3 "
                            "within 0.25, 4 within 0.1 (finest edge 1/128), 2:1 balanced, 17,528 leaves in Z "
                            "order, 60x60 trapezoid velocities on [-4,8]x[-6,6], T_w=1",
    "sphere_96_tree": "3D sphere r=0.5 at Ma 0.5, Kn 0.1 on an octree: a 32^3 root on [-4,4]^3 refined about the "
                      "centre to level 1 within 2.4 and 2 within 1.5 (finest edge 1/16), 2:1 balanced, 108,760 leaves "
                      "in Z order, 20^3 trapezoid velocities on [-5,5]^3",
    "batched_2d": "64 seeded 2D cases (seed 0): n ~ U{64..384} cells per axis on [-4,4]^2, m ~ U{16..40} "
                  "velocities per axis on [-6,6]^2, circle / ellipse (aspect U[1,3]) / NACA0012 (AoA U[0,10] deg), "
                  "Kn 10^U[-2,0], Ma U[0.1,0.8], mixed precision, one batch",
    "served": "Poisson request stream (seed 0, 20 requests/s): 80% 2D cases shaped like the batched workload, "
              "20% 3D spheres with 32..64 cells and 12..20 velocities per axis; continuous batching by HBM budget",
}


def _workload_case(args, workload, precision):
    """The case of a workload at the given precision (the cylinder at --kn)."""
    if workload == "cylinder_512":
        return WORKLOADS[workload](precision, args.kn)
    return WORKLOADS[workload](precision)


def kn_description(args, workload):
    d = DESCRIPTIONS[workload]
    return d.replace("Kn=0.1", f"Kn={args.kn:g}") if workload == "cylinder_512" else d


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere_96", choices=sorted(WORKLOADS))
    ap.add_argument("--kn", type=float, default=0.1,
                    help="cylinder_512: Knudsen number (the configuration sweeps 0.01, 0.1 and 1)")
    ap.add_argument("--no-nested", action="store_true",
                    help="sphere_96: skip the 512^2 cylinder measured in the same run")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--cells", type=int, default=0,
                    help="override the cells per axis, for tree workloads the root cells per axis (smaller cases for profiling captures)")
    ap.add_argument("--ncases", type=int, default=64, help="batched_2d: number of cases")
    ap.add_argument("--tune-steps", type=int, default=4,
                    help="batched_2d: steps per autotuner trial (0 = no tuning)")
    ap.add_argument("--nreq", type=int, default=16, help="served: number of requests")
    ap.add_argument("--serve-tol", type=float, default=1e-6, help="served: residual target")
    ap.add_argument("--serve-max-steps", type=int, default=20000, help="served: step cap per request")
    ap.add_argument("--fp64-nreq", type=int, default=6,
                    help="served: the sequential FP64 form runs the first N requests of the stream")
    ap.add_argument("--serve-round", type=int, default=20, help="served: steps per scheduling round")
    ap.add_argument("--no-fp64-serve", action="store_true", help="served: skip the sequential FP64 form")
    ap.add_argument("--error-report", type=int, default=0, metavar="STEPS",
                    help="instead of timing: run the workload STEPS steps in the mixed and the FP64 "
                         "GPU paths and print the relative differences of W, C_D, C_L, Q and the residual")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


BATCH_KERNEL = ("sweep2d_tma_batch_kernel", "paper_2512_20252_gb300/csrc/sweep_tma.cu")
L2_BYTES = 129 * 1000 * 1000  # GB300 L2 cache

SWEEP_KERNELS = {0: ("sweep_kernel", "paper_2512_20252_gb300/csrc/kernels.cu"),
                 1: ("sweep2d_tma_kernel", "paper_2512_20252_gb300/csrc/sweep_tma.cu"),
                 2: ("sweep3d_tma_kernel", "paper_2512_20252_gb300/csrc/sweep3d_tma.cu"),
                 3: ("tree_sweep_kernel", "paper_2512_20252_gb300/csrc/kernels.cu")}


def pinned_moments(torch, s):
    """Pinned host arrays for W^n and q^n of solver s (the end-to-end read)."""
    W = torch.empty((s.ncell, s.dim + 2), dtype=torch.float64, pin_memory=True).numpy()
    q = torch.empty((s.ncell, s.dim), dtype=torch.float64, pin_memory=True).numpy()
    return W, q


def profiled_traffic(kernel: str, source: str, pairs: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary (profiles/<kernel>_*.md, measured on a smaller case and scaled by
    the pairs processed), or None when the kernel source changed since."""
    import glob
    import hashlib

    try:
        sha = hashlib.sha1(open(os.path.join(ROOT, source), "rb").read()).hexdigest()
    except OSError:
        return None
    for path in glob.glob(os.path.join(ROOT, "profiles", kernel + "_*.md")):
        fields = {}
        for line in open(path):
            if ":" in line and line.split(":")[0] in ("traffic_bytes_per_pair", "source_sha1"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha1") == sha and "traffic_bytes_per_pair" in fields:
            return float(fields["traffic_bytes_per_pair"]) * pairs
    return None


# GB300's nominal FP64 rate (1.25 TFLOP/s dense, FMA = 2 flops), for context
# only: the FP64 path is reported against the rate measured on this GPU by
# ibdvm_fp64_fma_rate in the same run
FP64_NOMINAL_TFLOPS = 1.25


def profiled_fp64_flops_per_pair(dim: int):
    """FP64 operations per (cell, velocity) pair of the FP64 sweep (an FMA
    counted as two), from the committed ncu count of its executed FP64
    instructions (profiles/sweep_kernel_fp64_*.md), or None."""
    import glob

    for path in glob.glob(os.path.join(ROOT, "profiles", "sweep_kernel_fp64_*.md")):
        fields = {}
        for line in open(path):
            if ":" in line and line.split(":")[0] in ("fp64_flops_per_pair", "dim"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("dim") == str(dim) and "fp64_flops_per_pair" in fields:
            return float(fields["fp64_flops_per_pair"])
    return None


def max_over_ranks(x: float, pg, device: str = "cuda") -> float:
    """The largest x over all ranks (every rank gets it); x itself without a
    process group."""
    if pg is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_value(pairs_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the pairs every rank advanced (replicas of the
    same case) divided by the slowest rank's time."""
    return pairs_per_rank * steps * world / seconds


def dist_setup(nprocs: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_sample_case(case: dict) -> dict:
    """A bounded sample of the workload for the CPU oracle: the same gas,
    body, velocity grid and domain on a coarser cell grid (48 cells per axis in
    2D, 12 in 3D; a tree: the coarser tree the workload names, refined about
    the same centre or segment) so that one oracle step takes about a second."""
    c = dict(case)
    c["precision"] = "fp64"
    if case.get("tree"):
        from paper_2512_20252_gb300 import workloads

        spec = case["tree_spec"]
        smp = spec["sample"]
        c["n"] = list(smp["root"])
        if case["dim"] == 3:
            c["tree"] = workloads.tree_leaves_3d(tuple(smp["root"]), smp["maxlevel"], case["lo"], case["hi"],
                                                 spec["center"], smp["radii"])
        else:
            c["tree"] = workloads.tree_leaves(tuple(smp["root"]), smp["maxlevel"], case["lo"], case["hi"],
                                              spec["center"], smp["radii"], metric=spec.get("metric", "point"),
                                              segment=spec.get("segment"))
        return c
    c["n"] = [48] * 2 if case["dim"] == 2 else [12] * 3
    return c


def oracle_case(case: dict, threads: int):
    import oracle

    return oracle.OracleTree(case, threads=threads) if case.get("tree") else oracle.OracleCase(case, threads=threads)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(case: dict, budget_s: float, max_steps: int | None = None, threads: int = 1):
    import oracle

    oc = oracle_case(case, threads)
    oc.step(1)  # warm
    steps, t0 = 0, time.perf_counter()
    while True:
        oc.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps and steps >= max_steps) or (not max_steps and el > budget_s):
            break
    pairs = oc.nfluid * oc.nvel
    return pairs * steps / el, steps, el, oc


def cpu_baseline(sample: dict, budget_s: float, what: str) -> dict:
    """The oracle as it stands on a bounded sample of the workload, timed on all
    the host cores this process may use (OpenMP over ghosts and cells, bitwise
    the same results) and on one thread; `cores` is the thread count of the
    reported value."""
    nth = host_cores()
    v, n, el, oc = time_oracle(sample, budget_s, threads=nth)
    v1, n1, el1, _ = time_oracle(sample, budget_s / 2, threads=1)
    return {"value": v, "unit": "cell-velocity updates/s", "cores": nth, "kind": "oracle",
            "value_1thread": v1,
            "sample": f"{n} oracle steps ({el:.1f} s) on {nth} threads and {n1} ({el1:.1f} s) on one thread, "
                      f"of {what} on {sample['n'][0]} cells per axis ({oc.nfluid} fluid cells x {oc.nvel} velocities)"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    if args.workload == "batched_2d":
        case = batch_cases(args)[0]
    elif args.workload == "served":
        from paper_2512_20252_gb300 import workloads

        case = workloads.served_stream(0, nreq=1)[0][1]
    else:
        case = _workload_case(args, args.workload, args.precision)
    sample = cpu_sample_case(case)
    import oracle

    nth = host_cores()
    oc = oracle_case(sample, nth)
    for _ in range(max(args.warmup, 0)):
        oc.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oc.step(1)
    el = time.perf_counter() - t0
    pairs = oc.nfluid * oc.nvel
    value = pairs * args.steps / el
    desc = (f"oracle (plain FP64 C, {nth} host threads over ghosts and cells) on the workload's gas, body and "
            f"velocity grid with {sample['n'][0]} cells per axis")
    line = {
        "impl": "reference", "metric": "DVM cell x velocity updates/s", "value": value,
        "unit": "cell-velocity updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": kn_description(args, args.workload), "sample": desc},
        "cpu_baseline": {"value": value, "unit": "cell-velocity updates/s", "cores": nth, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "cell-velocity updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def error_report(args):
    """Mixed path (FP32 f, FP32 transport and relaxation with compensated
    sums, FP64 wall balance, forces and residual) against the FP64 path on the
    same workload; the FP64 path itself matches the CPU oracle within 1e-11
    (tests/test_parity_gpu.py)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)
    from paper_2512_20252_gb300 import ibdvm

    out = {}
    for prec in ("fp64", "mixed"):
        case = _workload_case(args, args.workload, prec)
        if args.cells and not case.get("tree"):
            case["n"] = [args.cells] * case["dim"]
        s = ibdvm.Solver(case, stream=torch.cuda.Stream().cuda_stream)
        res = s.step(args.error_report)
        W, q, t = s.moments()
        F, Q, CD, CL = s.forces()
        out[prec] = dict(W=W[t == 0], res=res, CD=CD, CL=CL, Q=Q, F=F)
        s.close()
    a, b = out["mixed"], out["fp64"]
    werr = [float(np.abs(a["W"][:, i] - b["W"][:, i]).max() / np.abs(b["W"][:, i]).max())
            for i in range(b["W"].shape[1])]
    rel = lambda x, y: float(abs(x - y) / max(abs(y), 1e-300))
    line = {"report": "mixed vs fp64", "workload": kn_description(args, args.workload), "steps": args.error_report,
            "W_rel_err": werr, "CD_rel_err": rel(a["CD"], b["CD"]), "CL_abs_err": abs(a["CL"] - b["CL"]),
            "Q_rel_err": rel(a["Q"], b["Q"]), "residual_rel_err": rel(a["res"], b["res"]),
            "fp64": {"CD": b["CD"], "CL": b["CL"], "Q": b["Q"], "residual": b["res"]},
            "mixed": {"CD": a["CD"], "CL": a["CL"], "Q": a["Q"], "residual": a["res"]}}
    print(json.dumps(line), flush=True)
    return 0


def batch_cases(args, precision="mixed"):
    from paper_2512_20252_gb300 import workloads

    cases = workloads.batched_2d(0, ncases=args.ncases, precision=precision)
    if args.cells:  # a smaller copy for profiling captures: cells per axis scaled down
        for c in cases:
            c["n"] = [max(16, c["n"][0] * args.cells // 384)] * 2
    return cases


def bench_batch(args, world, rank, local, pg):
    """The batched form: every case of the batch advanced by grouped launches
    (per step, one persistent sweep launch over the packed work list per chunk
    width of the members' velocity layouts)."""
    import numpy as np
    import torch

    from paper_2512_20252_gb300 import ibdvm

    cases = batch_cases(args)
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    solvers = [ibdvm.Solver(c, stream=stream.cuda_stream) for c in cases]
    batch = ibdvm.Batch(stream=stream.cuda_stream)
    for s in solvers:
        batch.add(s)
    setup_s = time.perf_counter() - t0
    pairs = sum(int(s.info.nfluid) * int(s.info.nvel) for s in solvers)
    alg_bytes = sum(int(s.info.nfluid) * int(s.info.nvel) * 2 * 4 * 2 for s in solvers)
    state_bytes = sum(int(s.ncell) * int(s.nvel_padded) * 2 * 4 for s in solvers)
    best_ms = batch.tune(args.tune_steps) if args.tune_steps else None
    tiling = batch.tiling()
    batch.step(max(args.warmup, 3))
    batch.set_profiling(True)
    batch.reset_kernel_times()
    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res, sts = batch.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    elapsed_ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop()
    kt = batch.kernel_times()
    batch.set_profiling(False)
    elapsed_ms = max_over_ranks(elapsed_ms, pg)
    value = job_value(pairs, args.steps, world, elapsed_ms / 1e3)
    # the sweep of one step is one persistent launch per chunk width of the
    # members' layouts, timed together: the roofline is per step
    sweep_ms, sweep_n = kt["sweep"]
    sweep_step_ms = sweep_ms / args.steps
    peak, peak_kind = peaks()
    achieved = alg_bytes / (sweep_step_ms / 1e3) / 1e9 if sweep_n else None
    launches = sum(n for _, n in kt.values())
    F, Q, CD, CL = batch.forces()

    # end to end through the C-ABI with host buffers: every step uploads each
    # member's f^n from pinned host memory, advances the batch one step and
    # reads every member's W^{n+1} back
    hbufs, outs = [], []
    for s in solvers:
        hb = torch.empty(s.native_shape(), dtype=torch.float32, pin_memory=True)
        s.get_f_native(hb.data_ptr(), hb.numel() * 4)
        hbufs.append(hb)
        outs.append(pinned_moments(torch, s))
    h2d = sum(hb.numel() * 4 for hb in hbufs)
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        for s, hb in zip(solvers, hbufs):
            s.set_f_native(hb.data_ptr(), hb.numel() * 4)
        batch.step(1)
        d2h = 0
        for s, (Wh, qh) in zip(solvers, outs):
            W, q, _ = s.moments(Wh, qh, with_types=False)
            d2h += W.nbytes + q.nbytes + 8
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, pg)
    e2e_value = job_value(pairs, e2e_steps, world, e2e_s)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cpu_sample_case(cases[0]), args.cpu_sample_seconds, "case 0's gas, body and velocity grid")
    if rank == 0:
        line = {
            "metric": "DVM cell x velocity updates/s", "value": value, "unit": "cell-velocity updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": DESCRIPTIONS["batched_2d"].replace("64 seeded", f"{args.ncases} seeded")
                       + (f", cells scaled by {args.cells}/384" if args.cells else ""),
                       "precision": "mixed", "cases": len(solvers), "pairs": pairs,
                       "state_gb": 2 * state_bytes / 1e9, "tiling": tiling, "tuned_ms_per_step": best_ms,
                       "setup_s": setup_s,
                       "l2": f"inputs larger than L2 (f^n is {state_bytes / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": profiled_traffic(BATCH_KERNEL[0], BATCH_KERNEL[1], pairs),
                         "kernel": BATCH_KERNEL[0], "peak_kind": peak_kind,
                         "alg_bytes_per_step": alg_bytes, "sweep_ms_per_step": sweep_step_ms,
                         "sweep_launches_per_step": sweep_n / args.steps},
            "kernel_ms": {k: v[0] for k, v in kt.items()},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "cell-velocity updates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "cpu_baseline": cpu, "clocks": clocks,
            "max_residual": float(np.max(res)), "statuses_ok": bool(np.all(sts == 0)),
            "CD_range": [float(np.min(CD)), float(np.max(CD))],
        }
        print(json.dumps(line), flush=True)
    batch.close()
    for s in solvers:
        s.close()
    return 0


def serve_stream(server, stream):
    """Drives a server with arrivals at their times; returns per-request
    (arrival, result) with times on the server's clock."""
    t_start = server.clock()
    pending = list(stream)
    ids = []
    active = queued = 0
    while pending or active or queued:
        now = server.clock() - t_start
        while pending and pending[0][0] <= now:
            t_arr, case = pending.pop(0)
            ids.append((t_arr, server.submit(case)))
        if not active and not queued and pending:
            time.sleep(max(0.0, pending[0][0] - (server.clock() - t_start)))
            continue
        active, queued, _ = server.poll()
    return [(t_start + t_arr, server.result(i)) for t_arr, i in ids]


def latency_stats(rows):
    import numpy as np

    lat = np.array([r["t_done"] - t for t, r in rows])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def bench_serve(args, rank):
    """Serving: the request stream through the batched server and, on the same
    stream, through the plain form (one request at a time, FP64 path)."""
    import numpy as np

    from paper_2512_20252_gb300 import ibdvm
    from paper_2512_20252_gb300 import workloads

    stream = workloads.served_stream(0, nreq=args.nreq, rate=20.0)

    def pairs_of(case):
        import math

        return math.prod(case["n"]) * math.prod(case["nv"])

    out = {}
    forms = [("batched_mixed", False, stream)]
    if not args.no_fp64_serve:
        forms.append(("sequential_fp64", True, stream[:max(1, min(args.fp64_nreq, len(stream)))]))
    for name, seq, reqs in forms:
        srv = ibdvm.Server(tol=args.serve_tol, max_steps=args.serve_max_steps, steps_per_round=args.serve_round,
                           sequential_fp64=seq)
        t0 = srv.clock()
        rows = serve_stream(srv, reqs)
        t1 = max(r["t_done"] for _, r in rows)
        srv.close()
        work = sum(pairs_of(c) * r["steps"] for (_, c), (_, r) in zip(reqs, rows))
        ok_rows = [(t, r) for t, r in rows if r["status"] == 0]
        out[name] = dict(latency_stats(ok_rows) if ok_rows else {}, makespan_s=t1 - t0, throughput=work / (t1 - t0),
                         requests=len(reqs),
                         converged=int(sum(r["status"] == 0 for _, r in rows)),
                         capped=int(sum(r["status"] == 6 for _, r in rows)),
                         failed=int(sum(r["status"] not in (0, 6) for _, r in rows)),
                         statuses=[int(r["status"]) for _, r in rows],
                         steps=[int(r["steps"]) for _, r in rows],
                         latency_s=[float(r["t_done"] - t) for t, r in rows],
                         CD=[float(r["CD"]) for _, r in rows], Q=[float(r["Q"]) for _, r in rows])
    b = out["batched_mixed"]
    line = {"metric": "served p50/p99 time-to-converge (s); throughput in cell-velocity updates/s",
            "value": b["throughput"], "unit": "cell-velocity updates/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "latency_p50_s": b.get("p50_s"), "latency_p99_s": b.get("p99_s"),
            "config": {"workload": DESCRIPTIONS["served"], "requests": args.nreq, "tol": args.serve_tol,
                       "max_steps": args.serve_max_steps, "steps_per_round": args.serve_round,
                       "offered_load_rps": 20.0, "work": "all cells x velocities x steps"},
            "forms": out}
    if "sequential_fp64" in out:
        f = out["sequential_fp64"]
        n = f["requests"]
        both = [i for i in range(n) if b["statuses"][i] == 0 and f["statuses"][i] == 0]
        line["vs_sequential_fp64"] = {
            "requests": n, "throughput_ratio": b["throughput"] / f["throughput"],
            "p99_ratio": (f["p99_s"] / b["p99_s"]) if "p99_s" in f and "p99_s" in b else None,
            "CD_max_rel_err_converged": max((abs(b["CD"][i] - f["CD"][i]) / max(abs(f["CD"][i]), 1e-300)
                                             for i in both), default=None),
            "steps_mixed_vs_fp64": [[b["steps"][i], f["steps"][i]] for i in range(n)]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    world, rank, local = dist_setup(args.gpus)
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.error_report:
        return error_report(args)

    import numpy as np
    import torch

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    pg = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
        if rank != 0:
            __graft_entry__.build()
        dist.barrier()
    torch.cuda.set_device(local)
    from paper_2512_20252_gb300 import ibdvm

    if args.workload in ("batched_2d", "served"):
        rc = bench_batch(args, world, rank, local, pg) if args.workload == "batched_2d" else bench_serve(args, rank)
        if pg:
            pg.barrier()
            pg.destroy_process_group()
        return rc
    line = measure_case(args, args.workload, world, rank, local, pg, with_cpu=not args.no_cpu_baseline)
    if (args.workload == "sphere_96" and not args.cells and args.precision == "mixed" and not args.no_nested):
        # the 2D configuration in the same run: 512^2 cells x 48^2 velocities,
        # then the tree-refined Ma 5 cylinder (value, roofline and end-to-end
        # figure of their own)
        sub = measure_case(args, "cylinder_512", world, rank, local, pg, with_cpu=False)
        if rank == 0:
            line["cylinder_512"] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "config", "roofline",
                                                      "kernel_ms", "gpu_launches", "e2e", "clocks", "residual",
                                                      "CD")}
            line["gpu_launches"] += sub["gpu_launches"]
        # the paper's Ma 5 cylinder on a tree-refined grid (69,148 leaves x 60^2)
        sub = measure_case(args, "cylinder_hypersonic_tree", world, rank, local, pg, with_cpu=False)
        if rank == 0:
            line["cylinder_hypersonic_tree"] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "config",
                                                                  "roofline", "kernel_ms", "gpu_launches", "e2e",
                                                                  "clocks", "residual", "CD")}
            line["gpu_launches"] += sub["gpu_launches"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


def measure_case(args, workload, world, rank, local, pg, with_cpu=True):
    """Times K steps of one workload on this rank's GPU (replicas on every
    rank) and returns the JSON line of rank 0 (None on the other ranks)."""
    import torch

    from paper_2512_20252_gb300 import ibdvm

    case = _workload_case(args, workload, args.precision)
    if args.cells and not case.get("tree"):
        case["n"] = [args.cells] * case["dim"]
    elif args.cells:
        # a tree workload with a smaller root grid (profiling captures)
        from paper_2512_20252_gb300 import workloads

        case = getattr(workloads, workload)(precision=args.precision, root=args.cells)
    stream = torch.cuda.Stream()
    solver = ibdvm.Solver(case, stream=stream.cuda_stream)
    if case.get("tree") and case["body"]["kind"] == "none":
        # no body on a tree: start from the freestream with a density bump of
        # 20% over the refined region, so that the steps do transport work
        import numpy as np

        from paper_2512_20252_gb300 import workloads

        xc = workloads.tree_centres(case)
        f = solver.get_f()
        f *= (1.0 + 0.2 * np.exp(-(xc[:, 0] ** 2 + xc[:, 1] ** 2) / 2.0))[:, None, None]
        solver.set_f(f)
        del f
    info = solver.info
    pairs = int(info.nfluid) * int(info.nvel)
    esize = 8 if args.precision == "fp64" else 4
    ncomp = int(info.ncomp)

    # warm-up (untimed)
    solver.step(max(args.warmup, 3))
    solver.set_profiling(True)
    solver.reset_kernel_times()
    sampler = ClockSampler(local)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    state_bytes = int(info.ncell) * int(info.nvel_padded) * ncomp * esize
    flush_l2 = state_bytes < L2_BYTES
    if flush_l2:
        # a state that fits in L2: one step at a time, L2 flushed by a write
        # of twice its size on the stream between the timed steps
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
        elapsed_ms = 0.0
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev0.record(stream)
            res = solver.step(1)
            ev1.record(stream)
            torch.cuda.synchronize()
            elapsed_ms += ev0.elapsed_time(ev1)
        del flush
    else:
        ev0.record(stream)
        res = solver.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed_ms = ev0.elapsed_time(ev1)
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    kt = solver.kernel_times()
    solver.set_profiling(False)
    elapsed_ms = max_over_ranks(elapsed_ms, pg)
    value = job_value(pairs, args.steps, world, elapsed_ms / 1e3)
    sweep_ms, sweep_n = kt["sweep"]
    kname, ksrc = SWEEP_KERNELS.get(int(info.sweep_variant), SWEEP_KERNELS[0])
    alg_bytes = pairs * ncomp * esize * 2  # read f^n, write f^{n+1}
    peak, peak_kind = peaks()
    achieved = alg_bytes / (sweep_ms / sweep_n / 1e3) / 1e9 if sweep_n else None
    launches = sum(n for _, n in kt.values())
    F, Q, CD, CL = solver.step_forces()

    # end to end through the C-ABI with host buffers: every step uploads f^n
    # from pinned host memory, advances one step and reads W^{n+1} back
    shp = solver.native_shape()
    hbuf = torch.empty(shp, dtype=torch.float32 if esize == 4 else torch.float64, pin_memory=True)
    nbytes = hbuf.numel() * esize
    solver.get_f_native(hbuf.data_ptr(), nbytes)
    Wh, qh = pinned_moments(torch, solver)
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        solver.set_f_native(hbuf.data_ptr(), nbytes)
        solver.step(1)
        W, q, _ = solver.moments(Wh, qh, with_types=False)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, pg)
    d2h = W.nbytes + q.nbytes + 8
    e2e_value = job_value(pairs, e2e_steps, world, e2e_s)

    cpu = None
    if rank == 0 and with_cpu:
        cpu = cpu_baseline(cpu_sample_case(case), args.cpu_sample_seconds, "the workload's gas, body and velocity grid")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": profiled_traffic(kname, ksrc, pairs),
                "kernel": kname, "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": sweep_ms / max(sweep_n, 1)}
    fpp = (profiled_fp64_flops_per_pair(int(info.dim))
           if args.precision == "fp64" and not case.get("tree") else None)
    if fpp and sweep_n:
        # the FP64 path is bound by GB300's FP64 arithmetic rate, not by HBM:
        # its roof is the FMA rate measured now on this GPU (clocks sampled)
        sampler = ClockSampler(local)
        sampler.start()
        peak64, peak_ms = ibdvm.fp64_fma_rate(20000, stream.cuda_stream)
        peak_clocks = sampler.stop()
        tf = fpp * pairs / (sweep_ms / sweep_n / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": peak64, "unit": "TFLOP/s",
                    "frac": tf / peak64, "traffic": profiled_traffic(kname, ksrc, pairs),
                    "kernel": kname, "peak_kind": "measured FP64 FMA rate (ibdvm_fp64_fma_rate)",
                    "peak_clocks": peak_clocks, "peak_ms": peak_ms, "nominal_fp64_tflops": FP64_NOMINAL_TFLOPS,
                    "fp64_flops_per_pair": fpp,
                    "hbm_achieved_gbs": achieved, "avg_launch_ms": sweep_ms / max(sweep_n, 1)}
    line = None
    if rank == 0:
        line = {
            "metric": "DVM cell x velocity updates/s",
            "value": value,
            "unit": "cell-velocity updates/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if esize == 4 else "f64",
            "data": "synthetic",
            "config": {"workload": kn_description(args, workload) + (f" at {args.cells} cells per axis" if args.cells else ""),
                       "precision": args.precision,
                       "cells": int(info.ncell), "fluid_cells": int(info.nfluid), "velocities": int(info.nvel),
                       "l2": (f"L2 flushed between timed steps (f^n is {state_bytes / 1e6:.0f} MB)" if flush_l2
                              else f"inputs larger than L2 (f^n is {state_bytes / 1e9:.2f} GB)"),
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "kernel_ms": {k: v[0] for k, v in kt.items()},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "cell-velocity updates/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps},
            "cpu_baseline": cpu,
            "clocks": clocks,
            "residual": res,
            "CD": CD if math.isfinite(CD) else None,  # none without a free stream
        }
    solver.close()
    if pg:
        pg.barrier()
    return line if rank == 0 else None




if __name__ == "__main__":
    sys.exit(main())
