#!/usr/bin/env python
"""Benchmark of the H^2 strong recursive skeletonisation solver on one B300.

One step = factorise the H^2 matrix in float32 (float64 top level) and solve with
float64 iterative refinement until the normwise backward error
||Ax-b|| / (||A|| ||x||) <= 1e-10, on the 1,048,576-point Fibonacci-sphere problem
(kernel 1/(4 pi r), leaf 128, eta 1, eps_lu 1e-5, one N(0,1) right-hand side).
``--workload uneven`` instead runs the uneven batch: independent Gaussian-kernel
systems (3D, leaf 64, eta 1, eps_lu 1e-6, 4 right-hand sides each, sizes
log-uniform in [--nmin, --nmax]) factorised and refined together as one forest;
with several GPUs the systems are split over the ranks (LPT by size).  Any other
family of ``h2gen.WORKLOADS`` (e.g. ``helmholtz3d``, ``lru3d``) runs as one system,
its size set by ``--size`` (rounded down to a full lattice where the family has one).

Prints one JSON line (rank 0).  ``value`` is the device time of a step with the
matrix and right-hand side resident in HBM; ``e2e`` repeats the step through the
C-ABI with host buffers (matrix upload and solution download inside the timing).
``--impl reference`` times the CPU oracle on a bounded sample of the same workload.
Several GPUs run independent replicas (a single system does not shard).
"""
from __future__ import annotations

import argparse
import functools
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve s at N=1M: mixed vs FP64 at bwd err≤1e-10; HBM/FLOP roofline %"
BERR_TOL = 1e-10
MAXIT = 50


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="sphere")
    p.add_argument("--n", "--size", dest="n", type=int, default=0,
                   help="override the problem size (testing only; spell it --size under torchrun, whose own "
                        "parser takes --n for an abbreviation of its options)")
    p.add_argument("--nrhs", type=int, default=0, help="override the number of right-hand sides")
    p.add_argument("--fp64-arm", type=int, default=1, help="also time the float64 factor arm once")
    p.add_argument("--e2e-steps", type=int, default=1)
    p.add_argument("--cpu-baseline", type=int, default=1)
    p.add_argument("--precision", default="auto", choices=["auto", "fp32", "tf32x3"],
                   help="reduced-precision arm: float32 factor with the Schur update on the FMA pipes "
                        "(fp32) or on the tensor cores as split TF32 (tf32x3); auto = tf32x3 for the "
                        "sphere, fp32 for the uneven batch (whose ill-conditioned systems need the "
                        "more accurate factor)")
    p.add_argument("--w-step", default="auto", choices=["auto", "triangular", "inverse"],
                   help="how the mixed arm applies D_RR^-1 in W_U, W_L and the diagonal solve: "
                        "auto = the library's default for the precision")
    p.add_argument("--nsys", type=int, default=64, help="uneven batch: number of systems")
    p.add_argument("--nmin", type=int, default=2048, help="uneven batch: smallest system")
    p.add_argument("--nmax", type=int, default=16384, help="uneven batch: largest system")
    p.add_argument("--mem-per-point-kb", type=float, default=240.0,
                   help="uneven batch: estimated device memory per point (H^2 data held twice, "
                        "factor and working arrays) for the sub-batch split")
    p.add_argument("--mem-budget-gb", type=float, default=0.0,
                   help="uneven batch: device memory a sub-batch may use (0 = 85%% of the GPU's)")
    p.add_argument("--matrix-cache", default="", help="load the H^2 matrix from this .npz if it exists, "
                   "else build and save it there (lets a profiler run skip the construction)")
    return p.parse_args()


# ------------------------------------------------------------------ distributed
def _dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    rank = int(os.environ.get("RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dist.init_process_group(backend)
    return dist, rank, ws


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ helpers
def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak of a B300: 148 SMs x 128 FP32 lanes x 2 flop per clock."""
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


def _traffic(kernel: str, algorithmic_bytes: float, steps: int):
    """DRAM bytes per step of ``kernel`` from the committed ncu summary
    (profiles/traffic.json: DRAM read+write over algorithmic bytes, measured on a
    smaller case of the same workload family and scaled by the algorithmic bytes of
    this run), or None when no capture of the current kernel exists."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f).get(kernel)
    if not t:
        return None
    return {"bytes_per_step": t["dram_over_algorithmic"] * algorithmic_bytes,
            "dram_over_algorithmic": t["dram_over_algorithmic"], "source": t["source"]}


def _problem(args, device):
    from h2gen import make_problem
    from h2gen.problems import load_problem, save_problem
    over = {} if not args.n else {"n": _lattice_size(args.workload, args.n)}
    if args.matrix_cache and os.path.exists(args.matrix_cache):
        return load_problem(args.matrix_cache, device)
    pb = make_problem(args.workload, device=device, **over)
    if args.matrix_cache:
        save_problem(pb, args.matrix_cache)
    return pb


def _problems(args, device, rank, ws):
    """(problems of this rank, description) for the chosen workload."""
    if args.workload != "uneven":
        pb = _problem(args, device)
        w = pb.workload
        return [pb], (f"{w.name} N={pb.A.n} leaf={w.leaf} eta={w.eta} eps_lu={w.tol} "
                      f"nrhs={args.nrhs or w.nrhs}")
    from h2gen import make_problem, uneven_sizes
    from paper_2509_11152_b300.shard import lpt_partition
    sizes = uneven_sizes(args.nsys, args.nmin, args.nmax)
    mine = lpt_partition(sizes, ws)[rank]
    pbs = [make_problem("gauss3d", device=device, n=sizes[s], seed=s) for s in mine]
    w = pbs[0].workload
    return pbs, (f"uneven batch: {args.nsys} gauss3d systems, N log-uniform in [{args.nmin}, {args.nmax}] "
                 f"(total {sum(sizes)}; this rank {len(mine)} systems, {sum(sizes[s] for s in mine)} points), "
                 f"leaf={w.leaf} eta={w.eta} eps_lu={w.tol} nrhs={args.nrhs or w.nrhs} each")


def _rhs(n, nrhs, device):
    import torch
    g = torch.Generator(device="cpu").manual_seed(0)
    b = torch.randn(n, nrhs, generator=g, dtype=torch.float64)
    return b.to(device)


# ------------------------------------------------------------------ oracle timing
def _lattice_size(workload: str, n: int) -> int:
    """Largest size <= n that the workload's point set admits (a square number of
    points for the 2D lattice, a cube for the 3D lattice)."""
    from h2gen import WORKLOADS
    dim = {"laplace2d": 2, "helmholtz3d": 3}.get(WORKLOADS[workload].family, 0)
    if not dim:
        return n
    side = int(round(n ** (1.0 / dim)))
    while side ** dim > n:
        side -= 1
    return side ** dim


@functools.lru_cache(maxsize=4)
def _sample_problem(workload: str, n: int):
    """The input of an oracle sample, built once per size (construction is not timed)."""
    from h2gen import make_problem
    return make_problem(workload, n=n)


def _oracle_sample(workload: str, n_sample: int):
    """Oracle factor + float64 refined solve (plain corrections until the backward
    error is <= 1e-10) of a smaller member of the workload's family, as it stands.
    Returns (seconds, N, corrections, berr, x, unrefined x, problem, b)."""
    from h2gen import rhs
    from oracle import dense, rs
    pb = _sample_problem(workload, _lattice_size(workload, n_sample))
    A = pb.A.numpy()
    b = rhs(A.n, pb.workload.nrhs, seed=0)
    t0 = time.perf_counter()
    Z = rs.factorize(A, pb.workload.tol, pb.norm_a)
    x = rs.solve(Z, b)
    x0 = x.copy()
    it = 0
    while True:
        r = b - dense.matvec(A, x)
        berr = float(np.max(np.linalg.norm(r, axis=0) / (pb.norm_a * np.linalg.norm(x, axis=0))))
        if berr <= BERR_TOL or it >= MAXIT:
            break
        x = x + rs.solve(Z, r)
        it += 1
    return time.perf_counter() - t0, A.n, it, berr, x, x0, pb, b


def _timed_oracle(workload: str, n_sample: int, threads: int):
    """_oracle_sample in a fresh Python process whose BLAS / OpenMP pools have `threads`
    threads (the oracle's own code is one Python thread; its parallelism is inside the
    BLAS / LAPACK calls, whose pool size is fixed when numpy loads)."""
    import tempfile
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = str(threads)
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "oracle.npz")
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", workload, str(n_sample), out],
                           env=env, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"oracle child failed:\n{r.stderr[-3000:]}")
        z = np.load(out)
        sec, ns, it, berr = float(z["sec"]), int(z["n"]), int(z["it"]), float(z["berr"])
        x, x0 = z["x"], z["x0"]
    pb = _sample_problem(workload, ns)
    from h2gen import rhs
    return sec, ns, it, berr, x, x0, pb, rhs(ns, pb.workload.nrhs, seed=0)


def _oracle_child(workload: str, n_sample: int, out: str) -> None:
    sec, ns, it, berr, x, x0, _, _ = _oracle_sample(workload, n_sample)
    np.savez(out, sec=sec, n=ns, it=it, berr=berr, x=x, x0=x0)


def _cpu_baseline(workload: str, n_full: int, n_sample: int) -> tuple[dict, tuple]:
    """The oracle timed (not extrapolated) on a bounded sample of the workload, at one
    BLAS thread and at every host core; value = the all-core time."""
    ncpu = os.cpu_count() or 1
    one = _timed_oracle(workload, n_sample, 1)
    allc = _timed_oracle(workload, n_sample, ncpu)
    sec1, ns, it, berr = one[:4]
    secn = allc[0]
    base = {"value": secn, "unit": "s", "cores": ncpu, "kind": "oracle", "n": ns,
            "value_1thread": sec1,
            "sample": f"oracle (float64 numpy, as it stands) factor + refined solve of the same family at "
                      f"N={ns} (the bench workload has N={n_full}): {secn:.1f} s with BLAS on {ncpu} threads, "
                      f"{sec1:.1f} s on 1 thread; {it} corrections, berr {berr:.1e}; measured, not scaled"}
    return base, allc


def run_reference(args, dist, rank, ws):
    if rank != 0:
        return
    from h2gen import WORKLOADS, uneven_sizes
    if args.workload == "uneven":
        sizes = uneven_sizes(args.nsys, args.nmin, args.nmax)
        family, n_full, n_sample = "gauss3d", sum(sizes), 4096
        w = WORKLOADS[family]
        full = (f"uneven batch: {args.nsys} gauss3d systems, N log-uniform in [{args.nmin}, {args.nmax}] "
                f"(total {n_full})")
    else:
        family = args.workload
        w = WORKLOADS[family]
        n_full = _lattice_size(family, args.n or w.n)
        n_sample = min(n_full, 16384)
        full = f"{w.name} N={n_full}"
    ncpu = os.cpu_count() or 1
    for _ in range(args.warmup):
        _timed_oracle(family, min(n_sample, 4096), ncpu)
    times = []
    info = None
    for _ in range(args.steps):
        res = _timed_oracle(family, n_sample, ncpu)
        times.append(res[0])
        info = res
    v = statistics.mean(times)
    ns = info[1]
    wdesc = (f"{w.name} N={ns} leaf={w.leaf} eta={w.eta} eps_lu={w.tol} nrhs={w.nrhs} "
             f"(the oracle's bounded sample of the {full} workload, timed at the size it ran)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wdesc, "precision": "float64 oracle"},
            "cpu_baseline": {"value": v, "unit": "s", "cores": ncpu, "kind": "oracle", "n": ns,
                             "sample": f"each step: oracle (as it stands) factor + refined solve at N={ns} "
                                       f"({info[2]} corrections, berr {info[3]:.1e}), BLAS on {ncpu} threads; "
                                       f"measured, not scaled"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _oracle_err(h, sample, prec, tol):
    """The mixed arm against the float64 oracle on the oracle's sample problem: the
    refined solutions (both at backward error <= 1e-10) and the unrefined solves (the
    reduced-precision factor against the oracle's float64 factor)."""
    import torch
    _, ns, _, _, x_or, x0_or, pb, b = sample
    M = h.h2_matrix_create(pb.A)
    Z = h.h2_factor_create(M, tol, pb.norm_a, prec)
    bt = h.colmajor(torch.from_numpy(b).cuda())
    x = h.colmajor(torch.zeros_like(bt))
    it, berr, ok = h.h2_refine_solve(Z, M, bt, x, BERR_TOL, MAXIT)
    x0 = h.colmajor(torch.from_numpy(b).cuda())
    h.h2_solve(Z, x0)
    rel = float(np.linalg.norm(x.cpu().numpy() - x_or) / np.linalg.norm(x_or))
    rel0 = float(np.linalg.norm(x0.cpu().numpy() - x0_or) / np.linalg.norm(x0_or))
    return {"n": ns, "refined_vs_oracle_refined": rel, "solve_vs_oracle_solve": rel0, "iters": it,
            "berr": berr}


# ------------------------------------------------------------------ our arm
def _subbatches(args, rank, ws):
    """The uneven batch's systems of this rank split into sub-batches that fit the GPU
    (one bin when the whole share fits), with their sizes."""
    import torch
    from h2gen import uneven_sizes
    from paper_2509_11152_b300.shard import lpt_partition, memory_bins
    sizes = uneven_sizes(args.nsys, args.nmin, args.nmax)
    mine = lpt_partition(sizes, ws)[rank]
    budget = args.mem_budget_gb * 1e9 or 0.85 * torch.cuda.get_device_properties(0).total_memory
    cost = [sizes[s] * args.mem_per_point_kb * 1e3 for s in mine]
    return sizes, [[mine[k] for k in b] for b in memory_bins(cost, budget)]


def run_subbatched(args, dist, rank, ws, sizes, bins):
    """The uneven batch when one rank's share does not fit the GPU: its sub-batches are
    built, factorised and refined in turn (construction untimed), each timed with CUDA
    events over the same warm-up / steps as the whole-batch path; value = the sum of the
    sub-batches' step times (one pass over every system), max over ranks."""
    import torch
    from h2gen import make_problem
    import paper_2509_11152_b300 as h
    from paper_2509_11152_b300 import binding

    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    if args.precision == "auto":
        args.precision = "fp32"
    prec = h.H2_PREC_TF32X3 if args.precision == "tf32x3" else h.H2_PREC_FP32
    wflag = {"auto": 0, "triangular": binding.H2_FLAG_W_TRIANGULAR, "inverse": binding.H2_FLAG_W_INVERSE}[args.w_step]
    stream = torch.cuda.current_stream().cuda_stream
    total, setup_s, launches, refin = 0.0, 0.0, 0, []
    clocks = ClockSampler(dev_index)
    clocks.start()
    for b in bins:
        t0 = time.perf_counter()
        pbs = [make_problem("gauss3d", device="cuda", n=sizes[s], seed=s) for s in b]
        setup_s += time.perf_counter() - t0
        w = pbs[0].workload
        nrhs = args.nrhs or w.nrhs
        M = h.h2_matrix_create_batch([pb.A for pb in pbs])
        norms = [pb.norm_a for pb in pbs]
        n_tot = sum(pb.A.n for pb in pbs)
        del pbs
        torch.cuda.empty_cache()
        bv = h.colmajor(_rhs(n_tot, nrhs, "cuda"))
        x = h.colmajor(torch.zeros_like(bv))

        def step():
            Z = h.h2_factor_create(M, w.tol, norms, prec, stream=stream, flags=wflag)
            x.zero_()
            res = h.h2_refine_solve(Z, M, bv, x, BERR_TOL, MAXIT)
            del Z
            return res

        for _ in range(max(args.warmup, 0)):
            step()
        torch.cuda.synchronize()
        _barrier(dist)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = binding.lib().h2_kernel_launch_count()
        e0.record()
        for _ in range(args.steps):
            it, berr, ok = step()
        e1.record()
        torch.cuda.synchronize()
        launches += binding.lib().h2_kernel_launch_count() - l0
        total += e0.elapsed_time(e1) / 1e3 / args.steps
        refin.append({"systems": len(b), "points": n_tot, "iters": it, "berr": berr, "converged": ok})
        del M, bv, x
        torch.cuda.empty_cache()
    clk = clocks.stop()
    value = _max_over_ranks(dist, total)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
                "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"uneven batch: {args.nsys} gauss3d systems, N log-uniform in "
                                       f"[{args.nmin}, {args.nmax}] (total {sum(sizes)}), run as "
                                       f"{len(bins)} sub-batches on rank 0",
                           "precision": args.precision, "w_step": args.w_step,
                           "parallelism": f"systems split over {ws} GPUs (LPT), sub-batches by memory",
                           "l2": "inputs larger than L2", "setup_s": round(setup_s, 1)},
                "refinement": {"sub_batches": refin, "converged": all(r["converged"] for r in refin)},
                "clocks": clk, "gpu_launches": int(launches),
                "roofline": None, "e2e": None,
                "note": "sub-batched run: no per-kernel roofline, e2e or CPU baseline (the whole-batch path "
                        "reports them)"}
        print(json.dumps(line), flush=True)


def run_ours(args, dist, rank, ws):
    import torch
    from paper_2509_11152_b300 import build
    build.build()
    import paper_2509_11152_b300 as h
    from paper_2509_11152_b300 import binding

    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    if args.workload == "uneven":
        sizes, bins = _subbatches(args, rank, ws)
        if len(bins) > 1:
            return run_subbatched(args, dist, rank, ws, sizes, bins)
    t0 = time.perf_counter()
    pbs, desc = _problems(args, "cuda", rank, ws)
    As = [pb.A for pb in pbs]
    norms = [pb.norm_a for pb in pbs]
    norm_arg = norms[0] if len(norms) == 1 else norms
    w = pbs[0].workload
    nrhs = args.nrhs or w.nrhs
    n_tot = sum(A.n for A in As)
    setup_s = time.perf_counter() - t0
    M = h.h2_matrix_create_batch(As)
    torch.cuda.empty_cache()              # construction temporaries held by torch's cache
    b = h.colmajor(_rhs(n_tot, nrhs, "cuda"))
    x = h.colmajor(torch.zeros_like(b))
    stream = torch.cuda.current_stream().cuda_stream

    if args.precision == "auto":
        args.precision = "fp32" if args.workload == "uneven" else "tf32x3"
    prec_mixed = h.H2_PREC_TF32X3 if args.precision == "tf32x3" else h.H2_PREC_FP32
    wflag = {"auto": 0, "triangular": binding.H2_FLAG_W_TRIANGULAR, "inverse": binding.H2_FLAG_W_INVERSE}[args.w_step]

    def step(prec, flags=0):
        if prec == prec_mixed:
            flags |= wflag
        Z = h.h2_factor_create(M, w.tol, norm_arg, prec, stream=stream, flags=flags)
        x.zero_()
        it, berr, ok = h.h2_refine_solve(Z, M, b, x, BERR_TOL, MAXIT)
        return Z, it, berr, ok

    for _ in range(max(args.warmup, 0)):
        Z, it, berr, ok = step(prec_mixed)
        del Z
    torch.cuda.synchronize()
    clocks = ClockSampler(dev_index)
    clocks.start()
    _barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = binding.lib().h2_kernel_launch_count()
    e0.record()
    results = []
    kernel = {}
    for s in range(args.steps):
        Z, it, berr, ok = step(prec_mixed, flags=binding.H2_FLAG_TIME_KERNELS)
        results.append((it, berr, ok))
        st = h.h2_factor_stats_get(Z)
        for k, v in st["kernel_ms"].items():
            kernel.setdefault(k, [0.0, 0])
            kernel[k][0] += v
            kernel[k][1] += st["kernel_launches"][k]
        last_stats = st
        del Z
    e1.record()
    torch.cuda.synchronize()
    launches = binding.lib().h2_kernel_launch_count() - launches0
    _barrier(dist)
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    t_step = _max_over_ranks(dist, t_step)
    uneven = args.workload == "uneven"
    value = t_step        # batch: the ranks share one batch; otherwise N independent replicas

    # dominant factorisation kernel and its roofline
    peaks, peak_kind = _peaks()
    names = {"basis": "augment", "proj": "project", "schur": "schur", "lu": "lu_trsm", "trsm": "lu_trsm"}
    dom = max(kernel, key=lambda k: kernel[k][0])
    dom_ms = kernel[dom][0] / args.steps
    phase = names.get(dom)
    flops = last_stats["phase_flops"].get(phase, 0.0) if phase else 0.0
    bytes_ = last_stats["phase_bytes"].get(phase, 0.0) if phase else 0.0
    hbm = peaks["hbm_gbs"]
    if dom == "schur" and args.precision == "tf32x3":
        # split-TF32 tensor-core GEMM (3 TF32 MMAs per float32 product); TF32 peak = the
        # measured sustained bf16 peak x the nominal TF32 / bf16 ratio (1.1 / 2.25)
        cpeak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * (1.1 / 2.25) / 3.0
        cbound, csrc = "tensor", (" (tensor: 3xTF32 = measured sustained bf16 x 1.1/2.25 / 3)")
    else:
        cpeak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2032.0))
        cbound, csrc = "alu", " (alu: 148 SMs x 128 FP32 lanes x 2 x max SM clock)"
    ach_gbs = bytes_ / (dom_ms / 1e3) / 1e9 if dom_ms > 0 else 0.0
    ach_tf = flops / (dom_ms / 1e3) / 1e12 if dom_ms > 0 else 0.0
    ai = flops / bytes_ if bytes_ else float("inf")
    if ai * hbm / 1e3 < cpeak:        # bandwidth roof is the lower one
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm}
    else:
        roof = {"bound": cbound, "achieved": ach_tf, "peak": cpeak, "unit": "TFLOP/s", "frac": ach_tf / cpeak}
    roof.update({"kernel": dom, "ms_per_step": dom_ms, "launches_per_step": kernel[dom][1] / args.steps,
                 "algorithmic_flops": flops, "algorithmic_bytes": bytes_,
                 "compute_roof": {"bound": cbound, "peak_tflops": cpeak, "achieved_tflops": ach_tf,
                                  "frac": ach_tf / cpeak if cpeak else None},
                 "peak_source": "measured (MEASURED_PEAKS.json)" + (csrc if roof["bound"] != "hbm" else ""),
                 "traffic": _traffic("schur_tc" if dom == "schur" and args.precision == "tf32x3" else dom,
                                     bytes_, args.steps)})

    line = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "strong" if uneven else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": desc,
                       "precision": "float32 factor/solve" + (", Schur update on tcgen05 tensor cores as split "
                                     "TF32 (hi*hi + hi*lo + lo*hi)" if args.precision == "tf32x3" else "")
                                     + ", float64 top LU + refinement",
                       "w_step": args.w_step,
                       "parallelism": (f"systems split over {ws} GPUs (LPT)" if uneven else f"replicas x{ws}"),
                       "l2": "inputs larger than L2 (matrix "
                       f"{sum(A.nbytes() for A in As) / 1e9:.1f} GB)", "setup_s": round(setup_s, 1),
                       "csp": max(pb.stats["csp"] for pb in pbs), "kmax": max(pb.stats["kmax"] for pb in pbs)},
            "refinement": {"iters": [r[0] for r in results], "berr": [r[1] for r in results],
                           "converged": all(r[2] for r in results)},
            "phase_ms": {k: round(v, 2) for k, v in last_stats["phase_ms"].items()},
            "phase_gflop": {k: round(v / 1e9, 3) for k, v in last_stats["phase_flops"].items()},
            "phase_gbytes": {k: round(v / 1e9, 3) for k, v in last_stats["phase_bytes"].items()},
            "kernel_ms_per_step": {k: round(v[0] / args.steps, 2) for k, v in kernel.items()},
            "factor_host_ms": {k: round(v, 1) for k, v in last_stats["host_ms"].items()},
            "roofline": roof, "clocks": clk, "gpu_launches": int(launches)}

    # float64 factor arm (mixed vs float64 at the same backward error)
    if args.fp64_arm:                 # one timed step: the library is warm by now
        torch.cuda.synchronize()
        f0 = time.perf_counter()
        Z, it, berr, ok = step(h.H2_PREC_FP64)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - f0
        st64 = h.h2_factor_stats_get(Z)
        del Z
        line["fp64_arm"] = {"value": t64, "unit": "s", "iters": it, "berr": berr, "converged": ok,
                            "factor_ms": st64["factor_ms"], "speedup_mixed": t64 / t_step}

    # end to end through the C-ABI with host buffers
    if args.e2e_steps > 0:
        from dataclasses import replace
        Ahs = [replace(A, **{k: getattr(A, k).cpu().pin_memory() for k in ("U", "E", "S", "D")}) for A in As]
        bh = b.cpu().t().contiguous().pin_memory().t()           # column-major, pinned
        del M
        torch.cuda.synchronize()
        e2e = []
        for _ in range(args.e2e_steps):
            xh = torch.zeros_like(bh)
            torch.cuda.synchronize()
            f0 = time.perf_counter()
            Mh = h.h2_matrix_create_batch(Ahs, stream=stream)
            Z = h.h2_factor_create(Mh, w.tol, norm_arg, prec_mixed, stream=stream, flags=wflag)
            it, berr, ok = h.h2_refine_solve(Z, Mh, bh, xh, BERR_TOL, MAXIT)
            torch.cuda.synchronize()
            e2e.append(time.perf_counter() - f0)
            del Z, Mh
        idx_bytes = sum(np.asarray(getattr(A, k)).nbytes for A in As for k in
                        ("node_start", "node_size", "rank", "U_off", "E_off", "adm_ptr", "adm_col", "S_off",
                         "inad_ptr", "inad_col", "D_off"))
        h2d = sum(A.nbytes() for A in As) + idx_bytes + bh.numel() * 8
        e2e_v = _max_over_ranks(dist, statistics.mean(e2e))
        line["e2e"] = {"value": e2e_v, "unit": "s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(bh.numel() * 8)}

    if args.cpu_baseline and rank == 0 and ws == 1:
        base, sample = _cpu_baseline(w.name, n_tot, min(n_tot, 4096 if uneven else 16384))
        line["cpu_baseline"] = base
        line["oracle_err"] = _oracle_err(h, sample, prec_mixed, w.tol)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    if len(sys.argv) == 5 and sys.argv[1] == "--oracle-child":
        _oracle_child(sys.argv[2], int(sys.argv[3]), sys.argv[4])
        return
    args = _args()
    dist, rank, ws = _dist_init()
    try:
        if args.impl == "reference":
            run_reference(args, dist, rank, ws)
        else:
            run_ours(args, dist, rank, ws)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
