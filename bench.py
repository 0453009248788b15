#!/usr/bin/env python
"""Benchmark: milliseconds per optimisation iteration of density-based inverse
homogenization (6 periodic cell problems to relative residual 1e-5, C^H, objective,
sensitivities, filter adjoint and OC update) on one GB300.

One step = one optimisation iteration on a 512^3 cell (134.2M elements; bulk-modulus
objective, volume fraction 0.3, density filter radius 2, warm-started solves), the
configuration of the paper's headline 512^3 row. Inputs are synthetic (seeded
blurred-noise inclusion field), far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 512]

Under torchrun (N > 1) every rank solves its own cell (replicas, no collective on the
data path); rank 0 prints one JSON line with the max time over ranks.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PAPER_512_BULK_MS = 38030.0      # paper, 512^3 bulk vf 0.3: 38.03 s per iteration (GTX 1080Ti)
METRIC = "ms per opt. iteration at 256\u00b3/512\u00b3 (6 cases to rel-res 1e-5); stencil HBM GB/s"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--objective", default="bulk", choices=["bulk", "shear", "poisson", "logpoisson"])
    ap.add_argument("--vf", type=float, default=0.3)
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--max-iters", type=int, default=1000)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--sample-n", type=int, default=16, help="cell size of the reference arm's oracle sample")
    ap.add_argument("--second-n", type=int, default=256,
                    help="also time this cell size (5 steps after 3 warm-up); 0 = off")
    ap.add_argument("--profile-steps", type=int, default=5,
                    help="steps of the separate per-launch-timed replay that gives the kernel breakdown")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="finest-level smoothing sweeps before/after coarse correction (0 = library default, 1)")
    ap.add_argument("--coarse-sweeps", type=int, default=0,
                    help="sweeps before/after coarse correction on level 1 (0 = library default, 1)")
    ap.add_argument("--min-coarse", type=int, default=0,
                    help="coarsen while the next level keeps at least this many cells per axis (0 = library default, 4)")
    ap.add_argument("--sweep-growth", type=int, default=0,
                    help="factor by which each further level's sweeps grow, capped at 64 (0 = library default, 3)")
    ap.add_argument("--coarse-smoother", type=int, nargs=3, default=None,
                    metavar=("RESIDENT_MAX_N", "CLUSTER_MAX_N", "SPLIT_MAX_N"),
                    help="coarse Gauss-Seidel kernels: levels of at most RESIDENT_MAX_N cells per axis smooth as "
                         "one cluster launch per phase with the displacement in shared memory, at most "
                         "CLUSTER_MAX_N as one cluster launch through L2, at most SPLIT_MAX_N with a thread per "
                         "(vertex, case) (default: the library's)")
    ap.add_argument("--coarse-forms", action="store_true",
                    help="after the timed region, time one Gauss-Seidel sweep of every coarse level in each kernel "
                         "form and V-cycles under several form settings (the cell's own hierarchy)")
    ap.add_argument("--smoother", default="gs8", choices=["gs8", "chebyshev"])
    ap.add_argument("--sym", default="none", choices=["none", "reflect3", "rotate3", "reflect6"],
                    help="symmetry enforced on the sensitivity and the density every step")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "mixed"],
                    help="mixed: coarse-level stencils of the preconditioner stored in BF16")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--record-traffic", metavar="NCU_CSV",
                    help="write profiles/traffic.json from an ncu --csv capture of "
                         "dram__bytes_read.sum and dram__bytes_write.sum (one V-cycle's k_fine_gs "
                         "launches at --n) and exit")
    ap.add_argument("--traffic-command", default="", help="the capture command, stored beside the figure")
    ap.add_argument("--batch", type=int, default=0,
                    help="K > 0: the batched-cells workload instead, K cells of uneven size (n in "
                         "{32,48,64,96,128}, volume fraction 0.1-0.5, objectives bulk/shear/poisson), "
                         "each on its own stream, the 6K solves of a step in one lockstep batch")
    ap.add_argument("--graphs", action="store_true", help="replay CG iterations as CUDA graphs")
    ap.add_argument("--autotune", action="store_true",
                    help="time the fine Gauss-Seidel variants per cell size before the run and use the fastest")
    ap.add_argument("--warm-start", default="previous", choices=["previous", "learned", "delta"],
                    help="start of each solve: the previous iterate (default), the warm-start network's "
                         "prediction, or the previous iterate plus the predicted change since it")
    ap.add_argument("--compare-starts", action="store_true",
                    help="also replay the timed steps with the learned start (network trained in the setup) "
                         "and report both starts side by side")
    ap.add_argument("--train-n", type=int, default=64, help="cell size of the network's training snapshots")
    ap.add_argument("--train-cells", type=int, default=3)
    ap.add_argument("--train-iters", type=int, default=8, help="optimisation iterations per training cell")
    ap.add_argument("--train-steps", type=int, default=600)
    ap.add_argument("--train-lr", type=float, default=1e-3)
    ap.add_argument("--net-blocks", type=int, default=5)
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed harness
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ roofline bookkeeping
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# Algorithmic work per launch (average over the launches of a class in one V-cycle) of the
# finest-level kernel classes, N = n^3 vertices, 6 cases. Bytes: the DRAM traffic the
# operation implies at minimum; flops: the algorithm's arithmetic.
STENCIL_FLOP = (576 + 27 * 54) * 2      # 27 blocks from E and K0, applied to 6 cases
SOLVE_FLOP = 6 * 15 + 30                # 3x3 LDL^T and 6 solves


def algorithmic_work(kc: str, n: int, sweeps: int = 1):
    N = n ** 3
    if kc == "fine_gs":
        # colour pass: E 4N, the other colours' u 63N, f_c 9N, u_c 9N (85N); in the first
        # sweep from zero only lower colours are read (half: 53.5N). 1 of 2*sweeps sweeps.
        full_b, first_b = 85 * N, 53.5 * N
        full_f = (576 + 26 * 54 + SOLVE_FLOP) * 2 * N / 8
        first_f = (288 + 13 * 54 + SOLVE_FLOP) * 2 * N / 8
        w = 1.0 / (2 * sweeps)
        return w * first_b + (1 - w) * full_b, w * first_f + (1 - w) * full_f
    if kc == "fine_cheb":
        # degree 2: pointwise start (b 72, x 72, E 4), then three tiled steps reading the
        # iterate and b, one also the previous iterate, each writing the new iterate
        b = (148 + 216 + 216 + 288) / 4 * N
        f = ((72 * 2 + SOLVE_FLOP) + 3 * (STENCIL_FLOP + SOLVE_FLOP)) / 4 * N
        return b, f
    if kc == "fine_matvec":      # E 4N + p 72N + q 72N; difference form: 26 blocks + 468 sub
        return 148 * N, ((576 + 26 * 54) * 2 + 26 * 18) * N
    if kc == "fine_residual":    # V-cycle residual: E 4N + x 72N + b 72N + out 72N
        return 220 * N, STENCIL_FLOP * N
    if kc == "true_residual":    # f - K (u + ulo): E 4N + u 72N + ulo 72N + f 72N + out 72N
        return 292 * N, STENCIL_FLOP * N
    if kc == "element":          # u and ulo 144N, E (C^H) or rho and the output (sensitivity) 4N / 8N:
        # the class holds one launch of each, 150N on average; 6 x 576 + 21 x 24 FMA per element
        return 150 * N, (6 * 576 + 21 * 24) * 2 * N
    return None, None


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("fine_gs.cu", "stencil.cuh", "dev_common.cuh"):
        with open(os.path.join(ROOT, "paper_2301_08911_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kc: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, scaled to n^3; None if the
    kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kc)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e["dram_bytes_per_launch"] * (n ** 3) / (e["n"] ** 3)


# ------------------------------------------------------------------ CPU oracle sample
_ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle
from synthetic import smoothed_threshold_density
n, vf, kind, reps, method = {n}, {vf}, {kind!r}, {reps}, {method!r}
rho = smoothed_threshold_density(n, vf, {seed}).astype(np.float64)
times = []
for it in range(reps):
    t0 = time.perf_counter()
    out = oracle.optimization_iteration(rho, n, vf, kind, iteration=it, method=method, tol=1e-9)
    times.append(time.perf_counter() - t0)
    rho = out["rho_new"]
print(json.dumps({{"times_s": times}}))
"""

# the oracle's solve at each sample size: sparse LU at 16^3, its certified multigrid-
# preconditioned FP64 CG above (sparse LU at 32^3 takes tens of minutes)
ORACLE_METHOD = {16: "lu"}


def oracle_sample(n: int, vf: float, kind: str, reps: int, seed: int, procs: int = 1):
    """Time `reps` oracle iterations at n^3 in `procs` concurrent single-threaded processes
    (seeds seed, seed+1, ...). Returns (per-process lists of seconds, wall seconds)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[v] = "1"
    method = ORACLE_METHOD.get(n, "mgcg")
    t0 = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, "-c", _ORACLE_SNIPPET.format(
        root=ROOT, n=n, vf=vf, kind=kind, reps=reps, seed=seed + k, method=method)],
        stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=env) for k in range(procs)]
    outs = []
    for p in ps:
        so, se = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError(se[-2000:])
        outs.append(json.loads(so.strip().splitlines()[-1])["times_s"])
    return outs, time.perf_counter() - t0


def host_cpu() -> dict:
    """Core count and CPU model of the host the oracle runs on."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


def oracle_baseline(args, n_target: int) -> dict:
    """The FP64 oracle timed on this host: one thread at 16^3 (2 iterations) and 32^3 (one
    iteration), and all cores at once at 32^3 (one iteration per core, different seeds).
    The value in the metric's unit scales the measured 32^3 single-thread time by element
    count to n_target^3 (a lower bound: the oracle's CG iteration count grows with n); the
    measured sizes are reported as measured."""
    host = host_cpu()
    procs = max(1, min(int(host["nproc"] or 1), 64))
    t16, _ = oracle_sample(16, args.vf, args.objective, 2, args.seed)
    t32, _ = oracle_sample(32, args.vf, args.objective, 1, args.seed)
    tall, wall = oracle_sample(32, args.vf, args.objective, 1, args.seed, procs=procs)
    ms16 = 1000.0 * statistics.mean(t16[0])
    ms32 = 1000.0 * statistics.mean(t32[0])
    return {"value": ms32 * (n_target / 32) ** 3, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle (numpy/scipy; sparse LU at 16^3, certified multigrid-preconditioned CG "
                       f"to true relative residual 1e-9 at 32^3) optimisation iterations measured at 16^3 and 32^3 on this host; "
                       f"value = the 32^3 single-thread time x (n/32)^3 to {n_target}^3 (lower bound; "
                       f"256^3 and 512^3 are not run: the oracle's assembled K alone is 49 / 390 GB)"),
            "measured": {"16^3": {"ms_per_iteration": ms16, "threads": 1, "iterations": len(t16[0])},
                         "32^3": {"ms_per_iteration": ms32, "threads": 1, "iterations": 1},
                         "32^3_all_cores": {"ms_per_iteration": 1000.0 * wall / procs, "processes": procs,
                                            "threads_per_process": 1,
                                            "note": "throughput: one iteration per process, all at once"}},
            "host": host}


def workload_name(args):
    return (f"{args.n}^3 periodic hex8 cell, {args.objective} objective, volume fraction {args.vf}, "
            f"6 load cases to rel-res {args.tol:g}, filter radius 2, OC move 0.05 damping 0.5, "
            f"warm-started MG-PCG")


def config_dict(args):
    return {"workload": workload_name(args), "n": args.n, "elements": args.n ** 3,
            "objective": args.objective, "volfrac": args.vf, "rel_tol": args.tol,
            "density": f"seeded blurred-noise inclusions (seed {args.seed}), exactly vf solid",
            "l2": "inputs larger than L2 (18 planes x n^3 fp32 per field)",
            "parallelism": "replicas (one cell per GPU, no collective)",
            "symmetry": args.sym,
            "warm_start": {"previous": "previous iterate",
                           "learned": f"warm-start network trained at {args.train_n}^3 (pooled, prolonged)",
                           "delta": f"previous iterate + predicted change (network trained at {args.train_n}^3)"
                           }[args.warm_start],
            "precision": ("FP32 storage and arithmetic; double-float displacement and CG correction"
                          if args.precision == "fp32" else
                          "FP32 arithmetic; coarse-level stencils stored in BF16 (symmetrised); "
                          "double-float displacement and CG correction"),
            "smoother": ("8-colour block Gauss-Seidel" if args.smoother == "gs8" else "Chebyshev(2)/block-Jacobi")
                        + f", sweeps before+after the coarse correction: {args.sweeps or 1}+{args.sweeps or 1} on the "
                          f"finest level, {args.coarse_sweeps or 1}+{args.coarse_sweeps or 1} on level 1, growing "
                          f"{args.sweep_growth or 3}x per further level (at most 64)",
            "graphs": bool(args.graphs)}


# ------------------------------------------------------------------ coarse smoother forms
def coarse_forms(hom, n, stream, dev):
    """Device time of one 8-colour Gauss-Seidel sweep (homo_smooth) on every coarse level in
    each kernel form, and of one V-cycle (homo_vcycle) under several form settings, on the
    cell's own hierarchy and density; CUDA events on the context stream, 2 untimed and 20 (10
    V-cycles) timed repetitions. Random right-hand sides and iterates of the level's size."""
    import torch

    forms = {"vertex": (0, 0, 0), "item": (0, 0, 1024), "cluster": (0, 1024, 0), "resident": (1024, 1024, 0)}
    saved = hom.coarse_smoother()[:3]
    gen = torch.Generator(device=dev).manual_seed(11)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    sweep = {}
    level = 1
    while level + 1 < hom.num_levels:
        nl = n >> level
        f = torch.rand(18 * nl ** 3, device=dev, generator=gen) - 0.5
        u = torch.zeros_like(f)
        row = {}
        for name, sizes in forms.items():
            if name in ("cluster", "resident") and nl > 32:
                continue                       # one cluster per case: a few SMs for a large level
            hom.set_coarse_smoother(*sizes)
            row[name] = round(timed(lambda: hom.smooth(level, False, f, u), 20) * 1e3, 1)
        sweep[f"{nl}^3"] = row
        level += 1
    r = torch.rand(18 * n ** 3, device=dev, generator=gen) - 0.5
    r = (r.view(18, -1) - r.view(18, -1).mean(dim=1, keepdim=True)).reshape(-1).contiguous()
    z = torch.empty_like(r)
    vc = {}
    for sizes in [(0, 0, 0), (0, 16, 32), (16, 16, 32), tuple(saved), (8, 32, 32)]:
        hom.set_coarse_smoother(*sizes)
        vc[",".join(map(str, sizes))] = round(timed(lambda: hom.vcycle(r, z), 10), 3)
    hom.set_coarse_smoother(*saved)
    del r, z
    return {"sweep_us": sweep, "vcycle_ms": vc,
            "settings": "resident_max_n,cluster_max_n,split_max_n; library default " + ",".join(map(str, saved)),
            "note": "one homo_smooth sweep per level and form (the resident form times its shared-memory setup "
                    "once per sweep; inside a V-cycle it runs many sweeps per launch), then homo_vcycle"}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The oracle as it stands, timed on one host core for the same workload: each step is
    one oracle optimisation iteration of a --sample-n^3 sample (default 16^3, sparse LU) of
    the workload's generator, scaled by element count to the workload's n^3 (a lower
    bound: the oracle's cost grows faster than the element count)."""
    if rank != 0:
        return 0
    reps = args.warmup + args.steps
    sn = args.sample_n
    outs, _ = oracle_sample(sn, args.vf, args.objective, reps, args.seed)
    timed = outs[0][args.warmup:]
    scale = (args.n ** 3) / (sn ** 3)
    ms = 1000.0 * statistics.mean(timed) * scale
    method = ORACLE_METHOD.get(sn, "mgcg")
    sample = (f"FP64 oracle (numpy/scipy, {'sparse LU' if method == 'lu' else 'certified multigrid-preconditioned CG'}) "
              f"optimisation iterations at {sn}^3 (same generator, vf, objective), {args.steps} timed after "
              f"{args.warmup} warm-up, one thread, scaled by element count to {args.n}^3 (a lower bound)")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_dict(args),
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle", "sample": sample,
                             "measured_ms_per_iteration": {f"{sn}^3": 1000.0 * statistics.mean(timed)},
                             "host": host_cpu()},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ learned warm start
def train_warm_start(args, dev, stream):
    """Snapshots (filtered density, displacement) from short optimisation runs of other
    seeds at --train-n, then Adam steps of the warm-start network on them. Untimed setup."""
    import time

    import numpy as np
    import torch

    from paper_2301_08911_gb300 import binding
    from synthetic import conv_net_parameters, smoothed_threshold_density

    t0 = time.time()
    nt = args.train_n
    snaps = []
    for c in range(args.train_cells):
        hom = binding.Homogenization(nt, stream=stream.cuda_stream)
        r = torch.from_numpy(smoothed_threshold_density(nt, args.vf, 1000 + 17 * c)).to(dev)
        rt, sv, dc = torch.empty_like(r), torch.empty_like(r), torch.empty_like(r)
        for it in range(args.train_iters):
            hom.filter(2.0, r, rt)
            hom.set_density(rt)
            hom.solve_cases(args.tol, args.max_iters, warm_start=True, raise_on_noconv=False)
            u = torch.empty(18 * nt ** 3, device=dev)
            hom.get_displacement(u)
            snaps.append((rt.clone(), u))
            _, g = binding.objective(args.objective, hom.CH(), it, 0.8)
            hom.sensitivity(g, sv)
            hom.filter(2.0, sv, dc)
            hom.update(dc, r, args.vf)
        hom.close()
    torch.cuda.synchronize(dev)
    us = np.stack([u.cpu().numpy().astype(np.float64).reshape(6, -1) for _, u in snaps])
    s_u = np.sqrt((us ** 2).mean(axis=(0, 2))) / nt          # per-case displacement scale per cell size
    blocks = args.net_blocks
    shapes = binding.net_layer_shapes(blocks)
    params = conv_net_parameters(shapes, 4242, [1.0] + [1.0, 0.5] * blocks + [0.1])
    net = binding.WarmStartNet(blocks, params, stream=stream.cuda_stream)
    t1 = time.time()
    losses = []
    for step in range(args.train_steps):
        rt, u = snaps[step % len(snaps)]
        want = step < len(snaps) or step >= args.train_steps - len(snaps)
        l = net.train_step(nt, rt, u, nt * s_u, args.train_lr, want_loss=want)
        if want:
            losses.append(l)
    torch.cuda.synchronize(dev)
    # one network forward at the training size, timed with CUDA events on its stream
    u_tmp = torch.empty(18 * nt ** 3, device=dev)
    net.predict(nt, snaps[0][0], nt * s_u, u_tmp)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(stream)
    for _ in range(reps):
        net.predict(nt, snaps[0][0], nt * s_u, u_tmp)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = e0.elapsed_time(e1) / reps
    conv_flop = 2 * 27 * binding.NN_CHANNELS * (binding.NN_FEATURES + (2 * blocks + 1) * binding.NN_CHANNELS)
    fwd_tflops = conv_flop * nt ** 3 / (fwd_ms * 1e-3) / 1e12
    bf16_peak = None
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as fh:
            bf16_peak = json.load(fh).get("bf16_tflops")
    k = min(len(snaps), args.train_steps)
    info = {"train_n": nt, "snapshots": len(snaps), "adam_steps": args.train_steps, "lr": args.train_lr,
            "blocks": blocks, "channels": binding.NN_CHANNELS,
            "loss_first_epoch": float(np.mean(losses[:k])), "loss_last_epoch": float(np.mean(losses[-k:])),
            "forward_ms": round(fwd_ms, 4), "forward_conv_flop_per_voxel": conv_flop,
            "forward_tflops": round(fwd_tflops, 2),
            "forward_frac_of_measured_bf16": (round(fwd_tflops / bf16_peak, 4) if bf16_peak else None),
            "snapshot_s": round(t1 - t0, 2), "train_s": round(time.time() - t1, 3),
            "s_u": [round(float(v), 6) for v in s_u],
            "data": f"{args.train_cells} cells x {args.train_iters} optimisation iterations at {nt}^3, "
                    "seeds other than the benchmark cell's"}
    return net, s_u, info


class LearnedStart:
    """Sets the start of each solve from the warm-start network. The network runs on the
    density average-pooled to the training cell size (features span the same number of
    voxels as in training); its prediction is prolonged up the solver's own levels."""

    def __init__(self, args, hom, net, s_u, dev):
        import torch

        from paper_2301_08911_gb300 import binding
        self.b = binding
        self.mode, self.hom, self.net, self.n, self.nt = args.warm_start, hom, net, args.n, args.train_n
        f = self.n // self.nt
        if self.n % self.nt or f & (f - 1) or f.bit_length() > hom.num_levels:
            raise SystemExit("--train-n must be n / 2^k with k below the number of levels")
        self.L = f.bit_length() - 1                       # level of the training-size grid
        self.scale = self.n * s_u
        self.rc = torch.empty(self.nt ** 3, device=dev)
        self.rc_prev = torch.empty_like(self.rc) if self.mode == "delta" else None
        self.uc = torch.empty(18 * self.nt ** 3, device=dev)
        self.lev = [torch.empty(18 * hom.level_size(l) ** 3, device=dev) for l in range(1, self.L)]
        self.u = torch.empty(18 * self.n ** 3, device=dev)
        self.have_prev = False
        self.launches = 0

    def _up(self, add: bool):
        """uc on level L -> level 0 into self.u (overwrite or accumulate)."""
        if self.L == 0:
            return
        src = self.uc
        for l in range(self.L - 1, -1, -1):
            dst = self.u if l == 0 else self.lev[l - 1]
            if l == 0 and add:
                self.hom.prolong_add(0, src, dst)
            else:
                self.hom.prolong(l, src, dst)
            src = dst

    def __call__(self, rt):
        if self.L == 0:
            rc = rt                                       # same grid: no pooling
        else:
            self.b.nn_pool(self.n, self.n // self.nt, rt, self.rc)
            self.launches += 1
            rc = self.rc
        target = self.uc if self.L else self.u
        if self.mode == "learned":
            self.net.predict(self.nt, rc, self.scale, target)
            self._up(add=False)
            self.hom.set_displacement(self.u)
        elif self.have_prev:                             # delta: u_prev + P(rc) - P(rc_prev)
            if self.L:
                self.net.predict(self.nt, rc, self.scale, self.uc)
                self.net.predict(self.nt, self.rc_prev, -self.scale, self.uc, accumulate=True)
                self.hom.get_displacement(self.u)
                self._up(add=True)
            else:
                self.hom.get_displacement(self.u)
                self.net.predict(self.nt, rc, self.scale, self.u, accumulate=True)
                self.net.predict(self.nt, self.rc_prev, -self.scale, self.u, accumulate=True)
            self.hom.set_displacement(self.u)
        if self.mode == "delta":
            self.rc_prev.copy_(rc)                        # device-to-device copy of n_t^3 floats
            self.have_prev = True


# ------------------------------------------------------------------ our arm
STENCIL_CLASSES = ("fine_matvec", "fine_residual", "fine_gs", "true_residual")


def roofline_of(kc: str, kn: int, kms: float, n: int, sweeps: int, peak_hbm: float, peak_src: str,
                alu_peak: float, alu_src: str):
    """Roofline entry of a kernel class from its launch count and summed event time."""
    nbytes, nflops = algorithmic_work(kc, n, sweeps)
    if nbytes is None or kn <= 0:
        return None
    avg_s = kms / kn / 1000.0
    t_hbm = nbytes / (peak_hbm * 1e9)
    t_alu = nflops / (alu_peak * 1e12)
    gbs = nbytes / avg_s / 1e9
    tfl = nflops / avg_s / 1e12
    traffic = recorded_traffic(kc, n)
    base = {"kernel": kc, "avg_launch_ms": kms / kn, "launches": kn, "bytes_per_launch": nbytes,
            "flops_per_launch": nflops, "traffic": traffic, "hbm_gbs": gbs, "hbm_frac": gbs / peak_hbm,
            "alu_tflops": tfl, "alu_frac": tfl / alu_peak}
    if t_hbm >= t_alu:
        return dict(bound="hbm", achieved=gbs, peak=peak_hbm, unit="GB/s", frac=gbs / peak_hbm,
                    peak_source=peak_src, **base)
    return dict(bound="alu", achieved=tfl, peak=alu_peak, unit="TFLOP/s", frac=tfl / alu_peak,
                peak_source=alu_src, **base)


class Loop:
    """The optimisation loop of Sec. 5.2 on one cell, with exact snapshots of everything a
    step carries to the next (density, iteration counter, both parts of the displacement,
    the learned start's previous pooled density), so passes can replay the same steps."""

    def __init__(self, args, n, seed, stream, dev, warm_start="previous"):
        import torch

        from paper_2301_08911_gb300 import binding
        from synthetic import smoothed_threshold_density
        self.b, self.args, self.n, self.stream, self.dev = binding, args, n, stream, dev
        self.hom = binding.Homogenization(n, sweeps=args.sweeps, stream=stream.cuda_stream,
                                          smoother=args.smoother, precision=args.precision,
                                          coarse_sweeps=args.coarse_sweeps, sweep_growth=args.sweep_growth,
                                          min_coarse=args.min_coarse,
                                          graphs=args.graphs)
        if args.coarse_smoother:
            self.hom.set_coarse_smoother(*args.coarse_smoother)
        self.r = torch.from_numpy(smoothed_threshold_density(n, args.vf, seed)).to(dev)
        self.rt = torch.empty_like(self.r)
        self.s = torch.empty_like(self.r)
        self.dc = torch.empty_like(self.r)
        self.it = 0
        self.cg, self.relres = [], []
        self.learned = None

    def step(self):
        a, hom = self.args, self.hom
        hom.filter(2.0, self.r, self.rt)
        hom.set_density(self.rt)
        if self.learned is not None:
            self.learned(self.rt)
        its, rel, _ = hom.solve_cases(a.tol, a.max_iters, warm_start=True, raise_on_noconv=False)
        C = hom.CH()
        f, g = self.b.objective(a.objective, C, self.it, 0.8)
        hom.sensitivity(g, self.s)
        hom.filter(2.0, self.s, self.dc)
        if a.sym != "none":
            hom.symmetrize(a.sym, self.dc, self.dc)
        hom.update(self.dc, self.r, a.vf)
        if a.sym != "none":
            hom.symmetrize(a.sym, self.r, self.r)
        self.it += 1
        self.cg.append(its)
        self.relres.append(max(rel))
        return f

    def launches(self):
        lr = self.learned
        return self.hom.launch_count + (lr.net.launch_count + lr.launches if lr else 0)

    def snapshot(self):
        import torch
        N18 = 18 * self.n ** 3
        snap = {"r": self.r.clone(), "it": self.it, "hi": torch.empty(N18, device=self.dev),
                "lo": torch.empty(N18, device=self.dev)}
        self.hom.save_displacement(snap["hi"], snap["lo"])
        lr = self.learned
        if lr is not None and lr.rc_prev is not None:
            snap["rc_prev"], snap["have_prev"] = lr.rc_prev.clone(), lr.have_prev
        return snap

    def restore(self, snap):
        self.r.copy_(snap["r"])
        self.it = snap["it"]
        self.hom.restore_displacement(snap["hi"], snap["lo"])
        if "rc_prev" in snap:
            self.learned.rc_prev.copy_(snap["rc_prev"])
            self.learned.have_prev = snap["have_prev"]
        self.cg, self.relres = [], []


def timed_steps(loop, steps, world, dev):
    """K steps between a barrier + synchronize on both sides, CUDA events on the stream."""
    import torch
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(loop.stream)
    for _ in range(steps):
        loop.step()
    e1.record(loop.stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    return max_over_ranks(e0.elapsed_time(e1), world)


def secondary_size(args, n2, stream, dev, world):
    """ms per optimisation iteration of a second cell size (the metric names 256^3 and
    512^3): 3 warm-up steps (the first cold), 5 timed, same workload otherwise."""
    import torch
    loop = Loop(args, n2, args.seed, stream, dev)
    cold = None
    for w in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop.step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if w == 0:
            cold = e0.elapsed_time(e1)
    loop.cg, loop.relres = [], []
    steps = 5
    t = timed_steps(loop, steps, world, dev)
    out = {"n": n2, "elements": n2 ** 3, "ms_per_step": t / steps, "steps": steps, "warmup": 3,
           "cold_first_iteration_ms": cold, "cg_iterations_per_step": [max(c) for c in loop.cg],
           "max_final_relres": max(loop.relres)}
    del loop
    torch.cuda.empty_cache()
    return out


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_2301_08911_gb300 import binding

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = args.n
    stream = torch.cuda.current_stream(dev)
    # measured FP32 peaks (scalar FMA and two-lane f32x2), the ALU roofline's denominators
    fp32_peak = {"scalar_tflops": binding.probe_fp32_peak(False), "f32x2_tflops": binding.probe_fp32_peak(True)}
    loop = Loop(args, n, args.seed + rank, stream, dev)
    hom = loop.hom
    tuning = None
    if args.autotune:
        hom.filter(2.0, loop.r, loop.rt)
        hom.set_density(loop.rt)
        choice, times = hom.autotune(retime=True)
        csizes, ctimes = hom.autotune_coarse(retime=True)
        tuning = {"cases_per_thread": choice[0], "threads_per_block": choice[1],
                  "ms_per_sweep": {f"{k[0]}x{k[1]}": round(v, 4) for k, v in times.items()},
                  "coarse_smoother": {"sizes": list(csizes),
                                      "ms_per_level_phase_pair": {f"{n >> lev}^3": {f: round(v, 4) for f, v in row.items()}
                                                                  for lev, row in ctimes.items()}}}
    net_info = None
    compare = None
    if args.warm_start != "previous" or args.compare_starts:
        net, s_u, net_info = train_warm_start(args, dev, stream)
        if args.warm_start != "previous":
            loop.learned = LearnedStart(args, hom, net, s_u, dev)
        else:
            compare = LearnedStart(argparse.Namespace(**{**vars(args), "warm_start": "learned"}), hom, net, s_u, dev)

    # warm-up (the first one is the cold solve from zero displacement)
    cold_ms = None
    for w in range(args.warmup):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop.step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if w == 0:
            cold_ms = e0.elapsed_time(e1)
    snap = loop.snapshot()
    loop.restore(snap)
    # kernels launched before the timed region (the probe's 16, the library's and the
    # snapshot's copy): the skip count of an ncu launch list of the timed steps
    launches_before = 16 + loop.launches() + 1

    # timed region: device time of K steps, no per-launch instrumentation
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = loop.launches()
    t_ms = timed_steps(loop, args.steps, world, dev)
    launches = loop.launches() - launches0
    clocks = sampler.stop()
    ms_step = t_ms / args.steps
    cg_timed = [list(c) for c in loop.cg]
    relres_timed = list(loop.relres)

    # end to end through the public API with host buffers, replaying the same K steps:
    # every step copies its density in from pinned host memory and the new density and C^H
    # out to the host
    e2e = None
    if not args.no_e2e:
        loop.restore(snap)
        host_rho = torch.from_numpy(loop.r.cpu().numpy()).pin_memory()
        barrier(world)
        torch.cuda.synchronize(dev)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(args.steps):
            loop.r.copy_(host_rho, non_blocking=True)
            loop.step()
            host_rho.copy_(loop.r, non_blocking=True)
        h1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(world)
        te = max_over_ranks(h0.elapsed_time(h1), world)
        e2e = {"value": te / args.steps, "unit": "ms", "h2d_bytes_per_step": 4 * n ** 3,
               "d2h_bytes_per_step": 4 * n ** 3 + 36 * 8,
               "note": "the same K steps as the timed region, replayed from an exact snapshot; density in "
                       "from and out to pinned host memory every step, C^H to the host",
               "replays_timed_steps": [list(c) for c in loop.cg] == cg_timed}

    # kernel breakdown: a separate replay of the timed steps with CUDA events around every launch
    prof_steps = min(args.steps, max(1, args.profile_steps))
    loop.restore(snap)
    torch.cuda.synchronize(dev)
    hom.profile(True)
    for _ in range(prof_steps):
        loop.step()
    prof = hom.profile_read()
    hom.profile(False)
    prof_same = [list(c) for c in loop.cg] == cg_timed[:prof_steps]

    # the same steps from the same snapshot with the learned start (timed the same way)
    starts = None
    if compare is not None:
        loop.restore(snap)
        loop.learned = compare
        t_l = timed_steps(loop, args.steps, world, dev)
        starts = {"previous": {"ms_per_step": ms_step, "cg_iterations_per_step": [max(c) for c in cg_timed]},
                  "learned": {"ms_per_step": t_l / args.steps,
                              "cg_iterations_per_step": [max(c) for c in loop.cg],
                              "max_final_relres": max(loop.relres)},
                  "note": "both replay the timed steps from the same snapshot; the learned start's time "
                          "includes pooling, the forward pass and the prolongation"}
        loop.learned = None

    forms = coarse_forms(hom, n, stream, dev) if args.coarse_forms else None

    second = None
    if args.second_n and args.second_n != n and world == 1:
        del snap
        torch.cuda.empty_cache()
        second = secondary_size(args, args.second_n, stream, dev, world)

    if rank != 0:
        return 0

    peak_hbm, peak_src = measured_peaks()
    sweeps = args.sweeps or 1
    alu_peak = fp32_peak["scalar_tflops"]
    alu_src = "measured: FP32 FMA probe (homo_probe_fp32_peak, scalar fma.rn.f32)"
    # the dominant kernel class among those with an algorithmic work model (the finest
    # level's stencil and smoother classes and the element kernel)
    modelled = {k: v for k, v in prof.items() if v[0] > 0 and algorithmic_work(k, n, sweeps)[0] is not None}
    roofline = None
    if modelled:
        dom = max(modelled.items(), key=lambda kv: kv[1][1])
        roofline = roofline_of(dom[0], dom[1][0], dom[1][1], n, sweeps, peak_hbm, peak_src, alu_peak, alu_src)
    stencil = {}
    for kc in STENCIL_CLASSES:
        kn, kms = prof.get(kc, (0, 0.0))
        r = roofline_of(kc, kn, kms, n, sweeps, peak_hbm, peak_src, alu_peak, alu_src)
        if r is not None:
            stencil[kc] = {k: r[k] for k in ("avg_launch_ms", "launches", "hbm_gbs", "hbm_frac", "alu_tflops",
                                             "alu_frac", "bytes_per_launch", "flops_per_launch", "bound")}

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(args, n)

    cg = np.array(cg_timed)
    line = {
        "metric": METRIC,
        "value": ms_step, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": (ms_step / PAPER_512_BULK_MS) if (n == 512 and args.objective == "bulk"
                                                          and abs(args.vf - 0.3) < 1e-9) else None,
        "dtype": "f32", "data": "synthetic", "config": config_dict(args),
        "roofline": roofline, "stencil": stencil, "fp32_peak": fp32_peak,
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
        "gpu_launches": launches, "launches_before_timed": launches_before,
        "solver": {"cold_first_iteration_ms": cold_ms,
                   "cg_iterations_per_step": cg.max(axis=1).tolist() if cg.size else [],
                   "max_final_relres": max(relres_timed) if relres_timed else None,
                   "coarse_smoother": dict(zip(("resident_max_n", "cluster_max_n", "split_max_n", "cluster",
                                                "resident_cluster"), hom.coarse_smoother()))},
        "kernels": {"steps": prof_steps, "replays_timed_steps": prof_same,
                    "note": "separate replay of the first timed steps with CUDA events around every launch",
                    **{k: {"launches": v[0], "ms": round(v[1], 3)} for k, v in prof.items() if v[0]}},
    }
    if second is not None:
        line["second_size"] = second
    if forms is not None:
        line["coarse_forms"] = forms
    if net_info is not None:
        line["warm_start"] = dict(mode=args.warm_start, **net_info)
    if starts is not None:
        line["start_comparison"] = starts
    if tuning is not None:
        line["autotune"] = tuning
    print(json.dumps(line), flush=True)
    return 0


def record_traffic(args) -> int:
    """Average DRAM bytes per launch of the fine Gauss-Seidel pass from an ncu CSV (the
    captured launches should be one V-cycle's 16 passes, first sweep included, which the
    roofline's algorithmic bytes average over too)."""
    import csv
    rows = list(csv.reader(open(args.record_traffic)))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[hi]
    ki, mi, vi, ui = h.index("Kernel Name"), h.index("Metric Name"), h.index("Metric Value"), h.index("Metric Unit")
    idx = h.index("ID") if "ID" in h else None
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    per = {}
    for r in rows[hi + 1:]:
        if len(r) <= vi or "k_fine_gs" not in r[ki]:
            continue
        if r[mi] in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            key = r[idx] if idx is not None else len(per)
            per[key] = per.get(key, 0.0) + float(r[vi].replace(",", "")) * scale[r[ui]]
    if not per:
        raise SystemExit("no k_fine_gs DRAM rows in " + args.record_traffic)
    path = os.path.join(ROOT, "profiles", "traffic.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    d["fine_gs"] = {"n": args.n, "launches": len(per), "dram_bytes_per_launch": sum(per.values()) / len(per),
                    "source_hash": kernel_source_hash(), "command": args.traffic_command}
    with open(path, "w") as fh:
        json.dump(d, fh, indent=1)
    print(json.dumps(d["fine_gs"]))
    return 0


def run_batch(args, rank, world, local):
    """K independent cells of uneven size per GPU, solved as one lockstep batch per step."""
    import numpy as np
    import torch

    from paper_2301_08911_gb300 import binding
    from synthetic import batched_cell_specs, smoothed_threshold_density

    torch.cuda.set_device(local)
    specs = batched_cell_specs(args.batch, args.seed + 100 * rank)
    cells = []
    for n, vf, obj, seed in specs:
        st = torch.cuda.Stream()
        hom = binding.Homogenization(n, stream=st.cuda_stream, graphs=args.graphs, precision=args.precision,
                                     coarse_sweeps=args.coarse_sweeps, sweep_growth=args.sweep_growth)
        if args.coarse_smoother:
            hom.set_coarse_smoother(*args.coarse_smoother)
        r = torch.from_numpy(smoothed_threshold_density(n, vf, seed)).cuda()
        cells.append({"hom": hom, "stream": st, "n": n, "vf": vf, "obj": obj, "r": r,
                      "rt": torch.empty_like(r), "s": torch.empty_like(r), "dc": torch.empty_like(r)})
    torch.cuda.synchronize()
    tuning = {}
    if args.autotune:
        for c in cells:
            c["hom"].filter(2.0, c["r"], c["rt"])
            c["hom"].set_density(c["rt"])
            choice, times = c["hom"].autotune()
            csizes, ctimes = c["hom"].autotune_coarse()
            if times:
                tuning[c["n"]] = {"cases_per_thread": choice[0], "threads_per_block": choice[1],
                                  "ms_per_sweep": {f"{k[0]}x{k[1]}": round(v, 4) for k, v in times.items()}}
            if ctimes:
                tuning.setdefault(c["n"], {})["coarse_smoother_sizes"] = list(csizes)
        torch.cuda.synchronize()
    it = {"k": 0, "cg": []}

    def step():
        for c in cells:
            c["hom"].filter(2.0, c["r"], c["rt"])
            c["hom"].set_density(c["rt"])
        its, rel, st = binding.solve_batch([c["hom"] for c in cells], args.tol, args.max_iters, warm_start=True)
        for c in cells:
            C = c["hom"].CH()
            f, g = binding.objective(c["obj"], C, it["k"], 0.8)
            c["hom"].sensitivity(g, c["s"])
            c["hom"].filter(2.0, c["s"], c["dc"])
            c["hom"].update(c["dc"], c["r"], c["vf"])
        it["k"] += 1
        it["cg"].append(int(its.max()))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    launches0 = sum(c["hom"].launch_count for c in cells)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    barrier(world)
    launches = sum(c["hom"].launch_count for c in cells) - launches0
    ms = max_over_ranks(1000.0 * (t1 - t0) / args.steps, world)
    if rank != 0:
        return 0
    elements = sum(n ** 3 for n, _, _, _ in specs)
    line = {"metric": "ms per batched optimisation iteration (uneven cells, 6 cases each to rel-res 1e-5)",
            "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.batch} cells per GPU, n in {{32,48,64,96,128}}, vf 0.1-0.5, "
                                   f"bulk/shear/poisson, lockstep batch solve"
                                   + (", CG iterations as CUDA graphs" if args.graphs else ""),
                       "cells": args.batch, "elements_per_gpu": elements,
                       "sizes": sorted({n for n, _, _, _ in specs}), "graphs": args.graphs,
                       "timing": "host clock around device-synchronised steps (one stream per cell)",
                       "autotune": tuning or None},
            "gpu_launches": launches, "solver": {"max_cg_iterations_per_step": it["cg"][-args.steps:]}}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.record_traffic:
        return record_traffic(args)
    rank, world, local = dist_setup()
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        if args.batch > 0:
            return run_batch(args, rank, world, local)
        return run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
