#!/usr/bin/env python
"""Benchmark of the deflated WaveHoltz solve on one B300 (replicas on N GPUs).

A step is one complete batched solve of the batched-squares workload: 256 problems -- constant-
speed Dirichlet squares of 257^2, 513^2, 769^2 and 1025^2 nodes x omega in {20, 30, 40, 50} x 16
Gaussian point sources of width 2h at seeded positions -- each deflated by its (grid, omega)'s 32
closed-form sine eigenvectors (DEVD, Algorithm 2; the 16 sources of one class share one basis),
solved by CG on (I - S_h) u = b to relative residual 1e-6, all problems advanced together: every
batched wave solve is ONE persistent launch, the CG loop a CUDA graph with a device-side WHILE
node.  Default precision: FP32 wave stepping inside FP64 residual correction (the b and residual
wave solves in double-float pairs, the Krylov and deflation arithmetic in FP64); the same line
carries the plain FP64 form's time on the same GPU (`fp64_form`), the 513^2 single-grid workload
(`c2`) and the HBM-resident 3-D stencil (`stencil_hbm`).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl whv|reference] [--workload c4|c2|...]

Prints one JSON line on rank 0.  --impl reference times the FP64 CPU oracle on the host cores
instead (a bounded sample per step, extrapolated to the whole workload with the oracle's own
iteration counts).  --gpus N without torchrun relaunches itself under torchrun with N ranks;
every rank solves its own copy of the workload (replicas: the path has no collective) and the
time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing
import os
import platform
import re
import socket
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the CPU oracle legs run one thread per process (numpy elementwise work is single-threaded
# anyway; this pins the BLAS calls of the projections too); set before numpy is first imported
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

METRIC = "WaveHoltz solve time to rel. residual 1e-6; stencil GLUP/s vs HBM roofline"
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2: written between timed steps of the L2-sized workloads


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="whv", choices=["whv", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="batched workload: skip the plain-FP64 form, c2, the 3-D stencil and e2e legs")
    ap.add_argument("--method", default="", choices=["", "cg", "dcg", "gmres", "agmres", "abicgstab"],
                    help="accelerator of the single-grid workloads (default: DCG for c1/c3, CG otherwise)")
    ap.add_argument("--steps-per-sweep", type=int, default=0,
                    help="2-D stepping kernel: 0 = autotune (default), k = blocked k steps per launch; "
                         "a fixed value keeps profiled runs on the kernel the plain run uses")
    ap.add_argument("--residual", default="df64", choices=["df64", "fp64"],
                    help="FP32 stepping: precision of the b and residual wave solves of the correction "
                         "(df64 = pairs of FP32 with error-free arithmetic; the accuracy check always uses FP64)")
    ap.add_argument("--check-every", type=int, default=1,
                    help="convergence test every k iterations; 1 keeps the CG loop on the device (a graph "
                         "with a conditional node), k > 1 launches one iteration graph per step from the host")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="FP32 stepping: relative reduction each inner CG solve of the correction aims for "
                         "(0 = the library default)")
    ap.add_argument("--eigs", default="lanczos", choices=["lanczos", "thick"],
                    help="variable-speed workload: one 1024-step Lanczos run, or thick-restart Lanczos (basis 3 nd + 4)")
    ap.add_argument("--lanczos-fp64", action="store_true",
                    help="variable-speed workload: FP64 stepping in the Lanczos eigen-solve (default: FP32)")
    ap.add_argument("--compress", type=float, default=0.0,
                    help="variable-speed workload: SVD-compress the basis with this Frobenius tolerance")
    ap.add_argument("--form", default="nonconservative", choices=["nonconservative", "conservative"],
                    help="variable-speed workload: operator form (conservative: div(c^2 grad), second order)")
    ap.add_argument("--sources", type=int, default=0,
                    help="batched workload: Gaussian sources per (grid, frequency) (default 16)")
    ap.add_argument("--workload", default="c4",
                    choices=["c1", "c2", "c3", "c4", "c4wave", "c5", "stencil3d", "study"],
                    help="c4 (default): the batched squares; c4wave: only the batched FP32 wave solve of those "
                         "problems (the dominant kernel, for profiling); c2: the 513^2 deflated solve; c1, c3, c5: "
                         "the 1-D, variable-speed 1025^2 and 3-D workloads; stencil3d: only the 256^3 FP32 wave "
                         "solves with one and two steps per launch (for profiling); study: iterations vs omega")
    return ap.parse_args(argv)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def relaunch_under_torchrun(args, argv):
    """--gpus N > 1 without a torchrun environment: run this script again as N ranks on this node
    (one replica per GPU) and return its exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", f"--master-port={_free_port()}", os.path.abspath(__file__), *argv]
    return subprocess.call(cmd)


def host_cpu():
    """Host cores this process may use and the CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = platform.processor() or ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"nproc": cores, "cpu_model": model}


# ------------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"], parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------ oracle legs
# The batched workload is far too large for the FP64 numpy oracle to solve within a benchmark run
# (about 10^12 lattice-point updates at ~5e7 per second and core).  Its time is therefore
# extrapolated from measured pieces of the oracle itself:
#   * the oracle's own iteration counts: DEVD-CG of every problem run to the workload's tolerance
#     by oracle/modal.py (the same CG in the box's sine eigenbasis, pinned to the time-domain
#     oracle: equal iteration counts up to rounding at the threshold);
#   * the time of one oracle CG iteration (one wave solve of krylov.Operator plus its vector
#     updates) on each grid size, per lattice-point update;
#   * for all host cores: the same CG iteration run by one process per core at once (the problems
#     are independent, so the oracle parallelises over them), which gives the aggregate rate.
# The oracle solve time of problem p is (iterations_p + 1) wave solves (the +1 is b) of
# N_p * Nt_p updates; the eigenvector set-up is left out on both sides (the GPU's timed step
# starts from bases that are already set, as the oracle's would).

def _c4_classes(nsrc):
    from paper_2606_31842_b300 import inputs as I
    return [(n, om) for n in I.C4_SIZES for om in I.C4_OMEGAS]


def _modal_iterations(job):
    """Oracle DEVD-CG iteration counts of the nsrc sources of one (grid, omega) class."""
    n, om, nsrc = job
    import numpy as np
    from oracle import operators as O, waveholtz as WH, modal as MD
    from paper_2606_31842_b300 import inputs as I
    w = I.WORKLOADS[f"c4_{n}_{int(om)}"]
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    ms = MD.ModalSystem(g, tg, w.nd)
    F = np.stack([I.forcing_for(w, s).reshape(g.shape) for s in range(nsrc)])
    its, conv, _ = MD.devd_cg(ms, F, w.tol, 20000)
    return {"n": n, "omega": om, "iterations": [int(x) for x in its], "converged": bool(conv.all()),
            "nt": tg.nt, "unknowns": g.n}


def _cg_iteration_time(job):
    """Seconds of one oracle CG iteration (krylov.cg, one step) on the class's grid and time grid,
    and the lattice-point updates of its wave solve."""
    n, om = job
    from oracle import operators as O, waveholtz as WH, krylov as K
    from paper_2606_31842_b300 import inputs as I
    w = I.WORKLOADS[f"c4_{n}_{int(om)}"]
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    b = I.random_field(g.shape, 7)
    A = K.Operator(g, tg)
    t0 = time.perf_counter()
    K.cg(g, A, b, 0.0, 1)
    t = time.perf_counter() - t0
    return {"n": n, "omega": om, "seconds": t, "lups": g.n * tg.nt}


def oracle_iterations(pool, nsrc):
    """Per-problem oracle iteration counts of the batched workload (in parallel over classes)."""
    jobs = [(n, om, nsrc) for n, om in _c4_classes(nsrc)]
    return pool.map(_modal_iterations, jobs, chunksize=1)


def oracle_time_model(classes, sec_per_lup, parallel_speedup):
    """Extrapolated oracle solve time (seconds) of the whole batch: sum over problems of
    (iterations + 1) wave solves at the measured seconds per update of their grid size."""
    total = 0.0
    lups = 0
    for c in classes:
        spl = sec_per_lup.get(c["n"], statistics.mean(sec_per_lup.values()))
        for it in c["iterations"]:
            total += (it + 1) * c["unknowns"] * c["nt"] * spl
            lups += (it + 1) * c["unknowns"] * c["nt"]
    return {"one_core_s": total, "all_cores_s": total / parallel_speedup, "lups": lups}


def oracle_parallel_speedup(pool, nworkers, job=(513, 50.0)):
    """All-core speed-up of the problem-parallel oracle: nworkers processes each run one oracle CG
    iteration at once (after a warm-up round); speed-up = nworkers x (time of the iteration run
    alone / its mean time when all run together), at most nworkers."""
    pool.map(_cg_iteration_time, [job] * nworkers, chunksize=1)          # warm-up round
    alone = min(pool.apply(_cg_iteration_time, (job,))["seconds"] for _ in range(2))
    t0 = time.perf_counter()
    res = pool.map(_cg_iteration_time, [job] * nworkers, chunksize=1)
    wall = time.perf_counter() - t0
    together = statistics.mean(r["seconds"] for r in res)
    return min(float(nworkers), nworkers * alone / together), wall


def oracle_c4_baseline(nsrc):
    """cpu_baseline of the batched workload: iteration counts, per-size update rates on one core
    (one CG iteration per grid size at omega = 50), all-core speed-up; about 30 s of host time."""
    cpu = host_cpu()
    P = cpu["nproc"]
    ctx = multiprocessing.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(P) as pool:
        classes = oracle_iterations(pool, nsrc)
        rates = pool.map(_cg_iteration_time, [(n, 50.0) for n in (257, 513, 769, 1025)], chunksize=1)
        speedup, wall_par = oracle_parallel_speedup(pool, P)
    spl = {r["n"]: r["seconds"] / r["lups"] for r in rates}
    model = oracle_time_model(classes, spl, speedup)
    return {"model": model, "classes": classes, "sec_per_lup": spl, "speedup": speedup, "cpu": cpu,
            "host_s": time.perf_counter() - t0}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the host cores, on the batched workload (or the
    513^2 workload with --workload c2).  Each timed step is a bounded sample: one oracle CG
    iteration on the next (grid, omega) class in turn (all 16 classes within 16 steps); `value`
    extrapolates the samples to the whole workload with the oracle's own iteration counts and the
    all-core speed-up, `ms_per_step` is the measured time of a sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload == "c2":
        return run_reference_c2(args)
    nsrc = args.sources if args.sources > 0 else 16
    cpu = host_cpu()
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(cpu["nproc"]) as pool:
        classes = oracle_iterations(pool, nsrc)
        speedup, _ = oracle_parallel_speedup(pool, cpu["nproc"])
    order = _c4_classes(nsrc)
    samples, step_ms = {}, []
    for s in range(args.warmup + args.steps):
        job = (257, 50.0) if s < args.warmup else order[(s - args.warmup) % len(order)]
        t0 = time.perf_counter()
        r = _cg_iteration_time(job)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            step_ms.append(dt * 1e3)
            samples.setdefault(r["n"], []).append(r["seconds"] / r["lups"])
    spl = {n: statistics.mean(v) for n, v in samples.items()}
    model = oracle_time_model(classes, spl, speedup)
    value = model["all_cores_s"] * 1e3
    nprob = sum(len(c["iterations"]) for c in classes)
    sample = (f"per step one oracle CG iteration (numpy FP64, 1 process) on the next of the 16 (grid, omega) "
              f"classes; extrapolated to all {nprob} problems with the oracle's own DEVD-CG iteration counts "
              f"(oracle/modal.py, tol 1e-6) and the measured {speedup:.1f}x speed-up of {cpu['nproc']} processes "
              f"(one problem per core); eigenvector set-up excluded on both sides")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": c4_config(nsrc, "DEVD-CG, FP64 (oracle)", nprob),
            "cpu_baseline": {"value": value, "unit": "ms", "cores": cpu["nproc"], "kind": "oracle",
                             "sample": sample, "cpu_model": cpu["cpu_model"],
                             "one_core_ms": model["one_core_s"] * 1e3, "parallel_speedup": speedup},
            "oracle_iterations_mean": statistics.mean(i for c in classes for i in c["iterations"]),
            "oracle_iterations_max": max(i for c in classes for i in c["iterations"]),
            "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def oracle_sample_c2(w, tol, iterations, budget_s=12.0):
    """The FP64 oracle on a bounded sample of the 513^2 workload: b and as many CG iterations as
    fit in the budget, extrapolated to `iterations`."""
    from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
    from paper_2606_31842_b300 import inputs as I
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    f = I.forcing_for(w)
    modes, lam2, _ = SP.select_modes(g, tg, w.nd)
    V = SP.basis(g, modes)
    t0 = time.perf_counter()
    b = WH.rhs_b(g, tg, K.project_out(g, V, f))
    t_b = time.perf_counter() - t0
    A = K.Operator(g, tg)
    k = max(1, int(budget_s / max(t_b, 1e-3)))
    t0 = time.perf_counter()
    K.cg(g, A, b, 0.0, k)
    t_it = (time.perf_counter() - t0) / k
    return {"solve_s": t_b + iterations * t_it, "t_wave": t_b, "t_iter": t_it, "k": k}


def oracle_iterations_c2(w, tol):
    """The oracle's DEVD-CG iteration count on the 513^2 workload (oracle/modal.py)."""
    import numpy as np
    from oracle import operators as O, waveholtz as WH, modal as MD
    from paper_2606_31842_b300 import inputs as I
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    its, conv, _ = MD.devd_cg(MD.ModalSystem(g, tg, w.nd), I.forcing_for(w).reshape(g.shape), tol, 20000)
    return int(its)


def run_reference_c2(args):
    from paper_2606_31842_b300 import inputs as I
    w = I.WORKLOADS["c2"]
    tol = 1e-6 if args.precision == "fp32" else w.tol
    iters = oracle_iterations_c2(w, tol)
    times, step_ms = [], []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        t = oracle_sample_c2(w, tol, iters, budget_s=2.0)
        if s >= args.warmup:
            times.append(t["solve_s"] * 1e3)
            step_ms.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.mean(times)
    cpu = host_cpu()
    cb = {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle", "cpu_model": cpu["cpu_model"],
          "sample": f"b + {t['k']} CG iterations per step (numpy FP64, 1 thread), extrapolated to the oracle's "
                    f"own {iters} DEVD-CG iterations (oracle/modal.py)"}
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": c2_config(w, tol, "fp64", None, args.gpus), "cpu_baseline": cb,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
# the sources a recorded traffic figure depends on: whole files, or (file, kernel) for the text of
# one kernel's definition in a file that holds others as well
KERNEL_SOURCES = {
    "k_block2d": ("stencil_blocked.cu", "quad2d.cuh", "whv_device.cuh"),
    "k_step3d": (("stencil.cu", "k_step3d"), "stencil_ops.cuh", "whv_device.cuh"),
    "k_step3d2": (("stencil.cu", "k_step3d2"), ("stencil.cu", "s3d2_plane"), "tma.cuh", "stencil_ops.cuh",
                  "whv_device.cuh"),
    "k_batch_block2d": (("batch.cu", "k_batch_block2d"), "quad2d.cuh", "whv_device.cuh"),
    "k_batch_tma": (("batch.cu", "k_batch_tma"), ("batch.cu", "tma_issue"), ("batch.cu", "tma_live_item"),
                    "quad2d.cuh", "tma.cuh", "whv_device.cuh"),
    "k_batch_front": (("batch.cu", "k_batch_front"), ("batch.cu", "front_clock"), ("batch.cu", "front_issue"),
                      ("batch.cu", "front_acc"), ("batch.cu", "wait_count"), "tma.cuh", "whv_device.cuh"),
}


def _kernel_text(src, name):
    """The definition of the __global__ kernel (or __device__ function) `name` in `src`: from its
    declaration to the closing brace of its body."""
    m = re.search(r"(?:__global__|__device__)[^;{]*?\b" + re.escape(name) + r"\(", src)
    if not m:
        raise KeyError(name)
    i = src.index("{", m.end())
    depth = 0
    for j in range(i, len(src)):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        if depth == 0:
            return src[m.start(): j + 1]
    raise ValueError(name)


def _code_only(text):
    """C/C++ source without its comments, whitespace runs made single spaces (edits of comments
    and layout do not change a kernel)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return re.sub(r"\s+", " ", text).strip()


def kernel_source_hash(kernel):
    """Hash of the code of one stepping kernel and the headers it uses (comments left out); a
    recorded DRAM traffic figure is only reported while the kernel is the one it was measured on."""
    h = hashlib.sha256()
    for item in KERNEL_SOURCES[kernel]:
        fn, name = item if isinstance(item, tuple) else (item, None)
        text = _code_only(open(os.path.join(ROOT, "paper_2606_31842_b300", "csrc", fn)).read())
        h.update((_kernel_text(text, name) if name else text).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel, precision):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the kernel
    source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(f"{kernel}:{precision}")
    except ValueError:
        return None
    if not rec:
        return None
    if kernel not in KERNEL_SOURCES or kernel_source_hash(kernel) != rec.get("source_sha"):
        return None
    return rec.get("dram_bytes_per_launch")


def aggregate_max(value, world, device=None):
    """Max of a per-rank time over all ranks (replicas: the job takes as long as its slowest rank);
    identity for a single process."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_max(value, world, device=None):
    """Max of a per-rank time over all ranks (replicas: the job takes as long as its slowest rank);
    identity for a single process."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _timed(stream, fn, steps, warmup, flush):
    import torch
    for _ in range(max(1, warmup)):
        fn()
    times, out = [], None
    for _ in range(steps):
        if flush is not None:
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    return statistics.mean(times), out


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(path)) if os.path.exists(path) else {}
    return peaks.get("hbm_gbs", 6400.0), ("measured" if "hbm_gbs" in peaks else "fallback")


def c4_config(nsrc, form, nprob):
    return {"workload": f"batched squares: (257, 513, 769, 1025)^2 nodes x omega (20, 30, 40, 50) x {nsrc} Gaussian "
                        f"point sources (width 2h, seeded), Dirichlet, c = 1, 32 closed-form eigenvectors per "
                        f"(grid, omega), {form}, to rel. residual 1e-6",
            "problems": nprob, "grids": [257, 513, 769, 1025], "omegas": [20.0, 30.0, 40.0, 50.0],
            "sources": nsrc, "nd": 32, "tol": 1e-6, "parallelism": "replicas (one batch per GPU)"}


class C4Batch:
    """The batched workload on the device: one grid per problem, the 16 sources of a (grid, omega)
    class sharing that class's closed-form basis; forcings resident on the device (and pinned on
    the host for the end-to-end leg)."""

    def __init__(self, whv, I, stream, fp32, nsrc, residual="df64", check_every=1, inner_tol=0.0):
        import torch
        self.whv, self.stream = whv, stream
        prec = whv.WHV_FP32_STEP if fp32 else whv.WHV_FP64
        self.grids, self.params, self.fs, self.hf, self.w = [], [], [], [], []
        t0 = time.perf_counter()
        for n in I.C4_SIZES:
            for om in I.C4_OMEGAS:
                w = I.WORKLOADS[f"c4_{n}_{int(om)}"]
                prm = whv.make_params(om, method="cg", tol=w.tol, maxit=3000, refine_fp64=fp32,
                                      residual_df64=fp32 and residual == "df64", check_every=check_every,
                                      inner_tol=inner_tol)
                owner = None
                for src in range(nsrc):
                    g = whv.Grid(w.npts, precision=prec, stream=stream)
                    if owner is None:
                        g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
                        owner = g
                    else:
                        g.whv_share_basis(owner)
                    h = torch.from_numpy(I.forcing_for(w, src).ravel()).pin_memory()
                    with torch.cuda.stream(stream):
                        self.fs.append(h.to("cuda", non_blocking=True))
                    self.grids.append(g); self.params.append(prm); self.hf.append(h); self.w.append(w)
        with torch.cuda.stream(stream):
            self.us = [torch.zeros(g.N, dtype=torch.float64, device="cuda") for g in self.grids]
        stream.synchronize()
        self.setup_s = time.perf_counter() - t0
        self.infos = None

    def solve(self):
        _, self.infos = self.whv.whv_solve_batched(self.grids, self.params, self.fs, self.us)
        return self.infos

    def close(self):
        for g in self.grids:
            g.close()
        self.grids = []


def batch_kernel_name(k):
    """The FP32 f = 0 batched 2-D kernel the library runs for k steps per sweep: the wavefront
    kernel for k = 8, the TMA-fed staged kernel for k = 4 and 12, k_batch_block2d otherwise (the
    library's diagnostic switch WHV_BATCH_TMA changes this: 0 = k_batch_block2d throughout, 1 or
    2 = the staged kernel for k = 4, 8, 12)."""
    env = os.environ.get("WHV_BATCH_TMA", "3")
    if env == "0" or k not in (4, 8, 12):
        return "k_batch_block2d"
    return "k_batch_front" if (k == 8 and env not in ("1", "2")) else "k_batch_tma"


def run_stencil3d(args):
    """--workload stencil3d: only the 256^3 FP32 f = 0 wave solves of the benchmark's stencil_hbm
    entry (whv_apply_pi, one and two leapfrog steps per launch); a small, self-contained command
    for ncu captures of k_step3d / k_step3d2."""
    import torch
    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    peak, _ = measured_peaks()
    line = stencil_hbm_measure(whv, torch.cuda.Stream(), peak)
    print(json.dumps({"metric": "3-D stencil step time", "unit": "us", "value": line["step_us"],
                      "higher_is_better": False, "stencil_hbm": line}))
    return 0


def run_c4wave(args):
    """--workload c4wave: only the batched FP32 f = 0 wave solve of the batched squares (one
    whv_apply_pi_batched launch per step, CUDA events), the kernel the solve spends most of its
    time in; a small, self-contained command for ncu captures."""
    import torch
    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    from paper_2606_31842_b300 import inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    nsrc = args.sources if args.sources > 0 else I.C4_SOURCES
    B = C4Batch(whv, I, stream, True, nsrc)
    if args.steps_per_sweep > 0:
        B.grids[0].whv_set_steps_per_sweep(args.steps_per_sweep)
        kb = args.steps_per_sweep
    else:
        kb = whv.whv_autotune_batched(B.grids, B.params)
    prm0 = [whv.make_params(p.omega) for p in B.params]
    outs = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in B.grids]
    vs = [torch.randn(g.N, dtype=torch.float64, device="cuda") for g in B.grids]

    def step():
        whv.whv_apply_pi_batched(B.grids, prm0, vs, None, outs)
    ms, _ = _timed(stream, step, args.steps, args.warmup, None)
    nts = [g.whv_time_grid(p)["nt"] for g, p in zip(B.grids, prm0)]
    lups = sum(g.N * nt for g, nt in zip(B.grids, nts))
    own = c4_sweep_bytes(B.grids, nts, kb)
    peak, _ = measured_peaks()
    print(json.dumps({"metric": "batched FP32 wave solve time", "value": ms, "unit": "ms", "steps": args.steps,
                      "warmup": args.warmup, "kernel": batch_kernel_name(kb), "steps_per_sweep": kb,
                      "problems": len(B.grids), "lups_per_launch": lups, "glups": lups / ms / 1e6,
                      "algorithmic_bytes_per_launch": own, "achieved_gbs": own / ms / 1e6,
                      "frac": own / ms / 1e6 / peak}), flush=True)
    B.close()
    return 0


def c4_sweep_bytes(grids, nts, k):
    """Algorithmic DRAM bytes of one FP32 f = 0 batched wave solve (k_batch_block2d, sweeps of k
    steps): per node, the first sweep reads v (8 B) and writes the state pair and the filter sum
    (12 B), every middle sweep reads and writes those three (24 B), the last one reads them and
    writes the FP64 output (20 B).  Halo re-reads are not counted."""
    total = 0
    for g, nt in zip(grids, nts):
        J = -(-nt // k)
        total += g.N * (20 + 24 * max(J - 2, 0) + (20 if J >= 2 else 0))
    return total


def c2_config(w, tol, precision, nt, n_gpus):
    return {"workload": f"2-D Helmholtz {w.npts[0]}x{w.npts[1]} nodes, omega={w.omega:g}, Gaussian source width 0.02, "
                        f"DEVD + CG with {w.nd} closed-form eigenvectors, tol {tol:g}",
            "grid": list(w.npts), "unknowns": w.n_unknowns, "omega": w.omega, "nd": w.nd, "tol": tol,
            "method": "DEVD-CG" + (" in FP64 residual correction" if precision == "fp32" else ""),
            "stepping": precision, "krylov": "fp64", "nt": nt,
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{n_gpus}"}


def c2_measure(whv, I, stream, flush, precision, steps, warmup, residual="df64", check_every=1, kfix=0):
    """The 513^2 workload: DEVD-CG solve time (CUDA events, L2 flushed between steps), the
    blocked kernel's equivalent bandwidth (its 3 MB state stays in L2) and the accuracy."""
    import torch
    w = I.WORKLOADS["c2"]
    fp32 = precision == "fp32"
    tol = 1e-6 if fp32 else w.tol
    g = whv.Grid(w.npts, precision=whv.WHV_FP32_STEP if fp32 else whv.WHV_FP64, stream=stream)
    prm = whv.make_params(w.omega, method="cg", tol=tol, maxit=5000, check_every=check_every,
                          refine_fp64=fp32, residual_df64=fp32 and residual == "df64")
    nt = g.whv_time_grid(prm)["nt"]
    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
    if kfix:
        g.whv_set_steps_per_sweep(kfix)
        ksweep = kfix
    else:
        ksweep = g.whv_autotune(prm)
    with torch.cuda.stream(stream):
        f = torch.from_numpy(I.forcing_for(w).ravel()).to("cuda")
        u = torch.zeros_like(f)
    res = {}

    def solve():
        res["info"] = g.whv_solve(prm, f, u)[1]
    ms, _ = _timed(stream, solve, steps, max(3, warmup), flush)
    info = res["info"]
    prm_chk = whv.make_params(w.omega, method="cg", tol=tol, maxit=5000, true_residual=True, refine_fp64=fp32,
                              residual_df64=fp32 and residual == "df64")
    _, ichk = g.whv_solve(prm_chk, f)
    # the step kernel alone: replays of the f = 0 wave-solve graph, per leapfrog step
    v = torch.randn(w.n_unknowns, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    torch.cuda.synchronize()
    g.whv_apply_pi(prm, v, None, out)
    stream.synchronize()
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.whv_apply_pi(prm, v, None, out)
    e1.record(stream)
    e1.synchronize()
    t_step = e0.elapsed_time(e1) * 1e-3 / (reps * nt)
    g.close()
    esz = 4 if fp32 else 8
    return {"solve_ms": ms, "tol": tol, "iterations": info["iterations"], "wave_solves": info["wave_solves"],
            "true_rel_residual": ichk["true_rel_residual"], "nt": nt, "steps_per_sweep": ksweep,
            "step_us": t_step * 1e6, "glups": w.n_unknowns / t_step / 1e9,
            "equiv_gbs": 5 * esz * w.n_unknowns / t_step / 1e9,
            "kernel": (f"k_block2d ({ksweep} leapfrog steps + filter per launch)" if ksweep > 1 else "k_step"),
            "note": "511^2 state (3 arrays, 3 MB) stays in the 126 MB L2: equivalent bandwidth, not an HBM figure"}


def stencil_hbm_measure(whv, stream, peak):
    """The 3-D 256^3 grid (66 MB per FP32 array, 3 arrays > L2): f = 0 wave solves with one
    (k_step3d) and two (k_step3d2) leapfrog steps per launch, the case on which the HBM fraction
    of the stencil is read."""
    import torch
    g3 = whv.Grid((256, 256, 256), precision=whv.WHV_FP32_STEP, stream=stream)
    prm3 = whv.make_params(40.0)
    nt3 = g3.whv_time_grid(prm3)["nt"]
    v3 = torch.randn(g3.N, dtype=torch.float64, device="cuda")
    o3 = torch.empty_like(v3)
    torch.cuda.synchronize()

    def time_3d(k):
        g3.whv_set_steps_per_sweep(k)
        g3.whv_apply_pi(prm3, v3, None, o3)
        stream.synchronize()
        reps3 = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps3):
            g3.whv_apply_pi(prm3, v3, None, o3)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / (reps3 * nt3)

    t31 = time_3d(1)
    t32 = time_3d(2)
    N = g3.N
    g3.close()
    ach31, ach32 = 20 * N / t31 / 1e9, 20 * N / t32 / 1e9
    return {"kernel": "k_step3d2 (3-D 7-point, two leapfrog steps + filter per launch, FP32)",
            "workload": "256^3 nodes (254^3 unknowns), omega=40, f = 0 wave solves, nt=%d" % nt3,
            "bound": "hbm", "achieved": ach32, "peak": peak, "unit": "GB/s", "frac": ach32 / peak,
            "bytes_per_lup": 20, "glups": N / t32 / 1e9, "step_us": t32 * 1e6,
            "own_bytes_per_lup": 12, "own_frac": 12 * N / t32 / 1e9 / peak,
            "traffic": traffic_for("k_step3d2", "fp32"), "traffic_unit": "DRAM bytes per launch (2 steps)",
            "note": "achieved/frac count the 20 B per LUP of single-step streaming (equivalent bandwidth); "
                    "own_frac counts the 12 B per LUP the two-step kernel must move",
            "single_step": {"kernel": "k_step3d (one step per launch)", "achieved": ach31, "frac": ach31 / peak,
                            "glups": N / t31 / 1e9, "step_us": t31 * 1e6, "traffic": traffic_for("k_step3d", "fp32")}}


def _env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _init_dist(world, local):
    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_c4(args):
    """The default line: the batched squares in one persistent launch per batched wave solve."""
    import torch
    rank, world, local = _env()
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    _init_dist(world, local)
    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    from paper_2606_31842_b300 import inputs as I
    stream = torch.cuda.Stream()
    nsrc = args.sources if args.sources > 0 else I.C4_SOURCES
    fp32 = args.precision == "fp32"
    B = C4Batch(whv, I, stream, fp32, nsrc, args.residual, args.check_every, args.inner_tol)
    if args.steps_per_sweep > 0:
        B.grids[0].whv_set_steps_per_sweep(args.steps_per_sweep)
        kb, ktag = args.steps_per_sweep, "fixed"
    else:
        kb, ktag = whv.whv_autotune_batched(B.grids, B.params), "autotuned"
    for _ in range(max(3, args.warmup)):
        B.solve()
    # ------------------------------------------------------------------ timed region
    times, infos = [], None
    launches0 = whv.whv_kernel_launches()
    with ClockSampler(local) as clk:
        time.sleep(0.5)                               # let the sampler start
        _barrier(world)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos = B.solve()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        _barrier(world)
    launches = whv.whv_kernel_launches() - launches0
    clocks = clk.summary()
    ms = aggregate_max(statistics.mean(times), world, device="cuda")
    nprob = len(B.grids)
    lups = sum(g.N * i["nt"] * i["wave_solves"] for g, i in zip(B.grids, infos))
    lups64 = sum(g.N * i["nt"] * i["wave_solves_fp64"] for g, i in zip(B.grids, infos))
    # FP64 true residual of a sample of the problems, recomputed on separate FP64 grids
    chk = []
    for p in range(0, nprob, 37):
        g64 = whv.Grid(B.w[p].npts, precision=whv.WHV_FP64, stream=stream)
        r = g64.whv_apply_pi(B.params[p], B.us[p], B.fs[p])
        bb = g64.whv_apply_pi(B.params[p], torch.zeros_like(B.fs[p]), B.fs[p])
        chk.append(float((r - B.us[p]).norm() / bb.norm()))
        g64.close()
    form = (("DEVD-CG with FP32 stepping inside FP64 residual correction"
             + (" (double-float b and residual wave solves)" if args.residual == "df64" else ""))
            if fp32 else "DEVD-CG, FP64 stepping")
    peak, peak_src = measured_peaks()
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if fp32 else "f64", "krylov_dtype": "f64", "data": "synthetic",
            "config": dict(c4_config(nsrc, form, nprob), steps_per_sweep=f"{kb} ({ktag})",
                           check_every=args.check_every, setup_s=B.setup_s,
                           l2="no flush: the working set (~1.5 GB of FP32 state, ~1 GB of forcings and "
                              "solutions) is larger than the 126 MB L2",
                           basis="one closed-form basis per (grid, omega), shared by its sources",
                           basis_bytes=sum(32 * I.WORKLOADS[f"c4_{n}_{int(om)}"].n_unknowns * 8
                                           for n in I.C4_SIZES for om in I.C4_OMEGAS),
                           basis_bytes_if_copied=sum(32 * g.N * 8 for g in B.grids),
                           contraction_bytes_per_projection=sum(
                               (32 + nsrc) * I.WORKLOADS[f"c4_{n}_{int(om)}"].n_unknowns * 8
                               for n in I.C4_SIZES for om in I.C4_OMEGAS),
                           contraction_bytes_per_projection_if_per_problem=sum((32 + 1) * g.N * 8 for g in B.grids)),
            "iterations_max": max(i["iterations"] for i in infos),
            "iterations_mean": statistics.mean(i["iterations"] for i in infos),
            "outer_iterations_max": max(i["outer_iterations"] for i in infos),
            "wave_solves": sum(i["wave_solves"] for i in infos),
            "wave_solves_fp64_or_df64": sum(i["wave_solves_fp64"] for i in infos),
            "glups_solve": lups / (ms * 1e-3) / 1e9, "lups_fp64_or_df64_share": lups64 / max(lups, 1),
            "accuracy": {"fp64_true_rel_residual_max": (max(i["true_rel_residual"] for i in infos) if fp32 else None),
                         "fp64_true_rel_residual_recomputed_sample_max": max(chk),
                         "recomputed": f"{len(chk)} problems, FP64 wave solves on separate FP64 grids"}}
    if not args.no_extras:
        # ---------------------------------------------------------------- e2e: host buffers
        # the same batched solve through the public API with the forcings copied from pinned host
        # memory and the solutions copied back inside the timed region (host wall clock, stream
        # synchronised at both ends)
        hu = [torch.empty(g.N, dtype=torch.float64).pin_memory() for g in B.grids]
        e2e = []
        for k in range(min(args.steps, 3) + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                for f, h in zip(B.fs, B.hf):
                    f.copy_(h, non_blocking=True)
            B.solve()
            with torch.cuda.stream(stream):
                for u, h in zip(B.us, hu):
                    h.copy_(u, non_blocking=True)
            stream.synchronize()
            if k > 0:
                e2e.append((time.perf_counter() - t0) * 1e3)
        nbytes = sum(g.N * 8 for g in B.grids)
        line["e2e"] = {"value": aggregate_max(statistics.mean(e2e), world, device="cuda"), "unit": "ms",
                       "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                       "timing": "host wall clock around H2D of every forcing, whv_solve_batched, D2H of every "
                                 "solution, stream synchronised"}
        del hu
        # ---------------------------------------------------------------- dominant kernel
        # k_batch_block2d (FP32, 5-point, c = 1): one batched f = 0 wave solve of all problems per
        # launch (whv_apply_pi_batched), timed with CUDA events on the launching stream
        if fp32:
            outs = [torch.empty(g.N, dtype=torch.float64, device="cuda") for g in B.grids]
            prm0 = [whv.make_params(p.omega) for p in B.params]
            whv.whv_apply_pi_batched(B.grids, prm0, B.us, None, outs)
            reps = 3
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                whv.whv_apply_pi_batched(B.grids, prm0, B.us, None, outs)
            e1.record(stream)
            e1.synchronize()
            t_launch = e0.elapsed_time(e1) * 1e-3 / reps
            nts = [i["nt"] for i in infos]
            lup_launch = sum(g.N * nt for g, nt in zip(B.grids, nts))
            own = c4_sweep_bytes(B.grids, nts, kb)
            kname = batch_kernel_name(kb)
            tr = traffic_for(kname, "fp32")
            tr_scaled = None
            if tr:
                rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[f"{kname}:fp32"]
                tr_scaled = tr * lup_launch / rec["lups_per_launch"]
            line["roofline"] = {"bound": "hbm", "achieved": own / t_launch / 1e9, "peak": peak, "unit": "GB/s",
                                "frac": own / t_launch / 1e9 / peak, "traffic": tr_scaled,
                                "kernel": f"{batch_kernel_name(kb)} ({kb} leapfrog steps + filter per sweep, all "
                                          f"{nprob} problems per launch)",
                                "algorithmic_bytes_per_launch": own, "lups_per_launch": lup_launch,
                                "launch_ms": t_launch * 1e3, "glups": lup_launch / t_launch / 1e9,
                                "equiv_single_step_gbs": 20 * lup_launch / t_launch / 1e9,
                                "peak_source": peak_src,
                                "note": "achieved counts the bytes the blocked kernel must move (3 FP32 reads and "
                                        "writes per node per sweep); equiv_single_step_gbs the 20 B per LUP of "
                                        "one-step streaming; traffic: ncu DRAM bytes of a smaller batch scaled by LUPs"}
            del outs
        # ---------------------------------------------------------------- plain FP64 form
        B64 = C4Batch(whv, I, stream, False, nsrc)
        k64 = whv.whv_autotune_batched(B64.grids, B64.params)
        warm = [whv.make_params(p.omega, method="cg", tol=p.tol, maxit=2) for p in B64.params]
        whv.whv_solve_batched(B64.grids, warm, B64.fs, B64.us)   # warm-up: kernels, graphs, FP64 buffers
        t64 = []
        for _ in range(1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            i64 = B64.solve()
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        ms64 = aggregate_max(statistics.mean(t64), world, device="cuda")
        line["fp64_form"] = {"ms": ms64, "speedup_of_value": ms64 / ms, "steps_per_sweep": k64,
                             "iterations_mean": statistics.mean(i["iterations"] for i in i64),
                             "iterations_max": max(i["iterations"] for i in i64),
                             "status": sorted(set(i["status"] for i in i64)),
                             "timing": "1 timed solve after a 2-iteration warm-up solve (CUDA events)"}
        B64.close()
        del B64
        # ---------------------------------------------------------------- c2 and the 3-D stencil
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        c2_32 = c2_measure(whv, I, stream, flush, "fp32", 10, 3, args.residual)
        c2_64 = c2_measure(whv, I, stream, flush, "fp64", 3, 3)
        line["c2"] = {"workload": c2_config(I.WORKLOADS["c2"], 1e-6, "fp32", c2_32["nt"], world)["workload"],
                      "fp32_correction": c2_32, "fp64": c2_64}
        del flush
        line["stencil_hbm"] = stencil_hbm_measure(whv, stream, peak)
    line["gpu_launches"] = launches
    line["clocks"] = clocks
    B.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_c4_baseline(nsrc)
        m = cb["model"]
        line["cpu_baseline"] = {
            "value": m["all_cores_s"] * 1e3, "unit": "ms", "cores": cb["cpu"]["nproc"], "kind": "oracle",
            "cpu_model": cb["cpu"]["cpu_model"], "one_core_ms": m["one_core_s"] * 1e3,
            "parallel_speedup": cb["speedup"], "host_s": cb["host_s"],
            "oracle_iterations_mean": statistics.mean(i for c in cb["classes"] for i in c["iterations"]),
            "sample": (f"numpy FP64 oracle: one CG iteration per grid size (omega = 50) on one core, the same "
                       f"iteration in {cb['cpu']['nproc']} processes at once for the all-core rate, the oracle's own "
                       f"DEVD-CG iteration counts of all {nprob} problems (oracle/modal.py); extrapolated to "
                       f"sum_p (iterations_p + 1) wave solves; eigenvector set-up excluded on both sides")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_c2(args):
    """--workload c2: the 513^2 deflated solve (FP32 + FP64 correction, or plain FP64 to 1e-8)."""
    import torch
    rank, world, local = _env()
    _init_dist(world, local)
    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    from paper_2606_31842_b300 import inputs as I
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    launches0 = whv.whv_kernel_launches()
    with ClockSampler(local) as clk:
        time.sleep(0.5)
        _barrier(world)
        r = c2_measure(whv, I, stream, flush, args.precision, args.steps, args.warmup, args.residual,
                       args.check_every, args.steps_per_sweep)
        _barrier(world)
    ms = aggregate_max(r["solve_ms"], world, device="cuda")
    w = I.WORKLOADS["c2"]
    peak, peak_src = measured_peaks()
    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "krylov_dtype": "f64",
            "data": "synthetic", "config": c2_config(w, r["tol"], args.precision, r["nt"], world),
            "c2": r, "gpu_launches": whv.whv_kernel_launches() - launches0, "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        iters = oracle_iterations_c2(w, r["tol"])
        cb = oracle_sample_c2(w, r["tol"], iters)
        line["cpu_baseline"] = {"value": cb["solve_s"] * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                                "sample": f"numpy FP64, 1 thread: b + {cb['k']} CG iterations, extrapolated to the "
                                          f"oracle's own {iters} DEVD-CG iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_workload(args):
    """The other workloads (one JSON line each): 1-D FP64 DCG, variable-speed 1025^2 with the device
    Lanczos basis, the 3-D cube and the omega study."""
    import numpy as np
    import torch
    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    from paper_2606_31842_b300 import inputs as I
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(a.ravel()).to("cuda")  # noqa: E731
    line = {"metric": METRIC, "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "data": "synthetic"}
    if args.workload == "study":
        # iterations vs omega with N_D growing linearly or quadratically in omega (Sec. 4.4):
        # DEVD-CG, FP64, closed-form vectors on the 257^2 unit square, omega = 10 .. 40
        res = {"quadratic": [], "linear": []}
        t_all = 0.0
        omegas = [10.0, 15.0, 20.0, 25.0, 30.0, 35.0, 40.0]
        for rule, nd_of in (("quadratic", lambda om: int(om * om // 10)), ("linear", lambda om: int(3 * om // 2))):
            for om in omegas:
                npts = (257, 257)
                g = whv.Grid(npts, precision=whv.WHV_FP64, stream=stream)
                prm = whv.make_params(om, method="cg", tol=1e-8, maxit=20000)
                g.whv_set_deflation_basis(prm, nd_of(om), whv.WHV_BASIS_CLOSED_FORM)
                f = dev(I.gaussian(npts, [0.37, 0.58], 1.0 / om, om * om))
                t0 = time.perf_counter()
                _, info = g.whv_solve(prm, f)
                t_all += time.perf_counter() - t0
                res[rule].append({"omega": om, "nd": nd_of(om), "iterations": info["iterations"],
                                  "status": info["status"]})
                g.close()
        line.update({"workload": "study", "value": t_all * 1e3, "ms_per_step": t_all * 1e3, "dtype": "f64",
                     "krylov_dtype": "f64",
                     "config": {"workload": "iterations vs omega on the 257^2 unit square, DEVD-CG to 1e-8 with "
                                            "N_D = floor(omega^2/10) (quadratic) or floor(3 omega/2) (linear) "
                                            "closed-form vectors; value = total solve time"},
                     "study": res})
        print(json.dumps(line), flush=True)
        return 0
    name = args.workload
    w = I.WORKLOADS["c5" if name == "c5" else name]
    prec = whv.WHV_FP64 if name == "c1" else whv.WHV_FP32_STEP
    cons = name == "c3" and args.form == "conservative"
    order = 2 if cons else w.order   # the conservative operator is second order
    g = whv.Grid(w.npts, order=order, precision=prec, stream=stream)
    if w.speed:
        c2v = dev(I.speed_squared(w.speed, w.npts, w.speed_seed))
        if cons:
            g.whv_set_speed_form(c2v, whv.WHV_SPEED_CONSERVATIVE)
        else:
            g.whv_set_speed(c2v)
    refine = prec == whv.WHV_FP32_STEP
    dfres = refine and args.residual == "df64" and not cons   # the conservative operator corrects in FP64
    method = args.method or ("dcg" if name in ("c1", "c3") else "cg")
    prm = whv.make_params(w.omega, method=method, tol=w.tol, maxit=20000, restart=30, refine_fp64=refine,
                          residual_df64=dfres)
    t0 = time.perf_counter()
    if name == "c3" and args.eigs == "thick":
        theta, resid, st = g.whv_lanczos_restarted(prm, w.nd, 3 * w.nd + 4, max_restarts=40, tol=1e-6,
                                                   fp64_stepping=args.lanczos_fp64)
        setup = {"basis": f"device thick-restart Lanczos on S_h ({'FP64' if args.lanczos_fp64 else 'FP32'} stepping, "
                          f"basis {3 * w.nd + 4}, tol 1e-6)",
                 "ritz_resid_median": float(np.median(resid)), "ritz_resid_max": float(np.max(resid)),
                 "setup_wave_solves": st["wave_solves"], "restarts": st["restarts"], "converged": st["converged"]}
    elif name == "c3":
        theta, resid = g.whv_lanczos(prm, w.nd, 1024, None, args.lanczos_fp64, 0)
        setup = {"basis": f"device Lanczos on S_h ({'FP64' if args.lanczos_fp64 else 'FP32'} stepping, 1024 steps)",
                 "ritz_resid_median": float(np.median(resid)), "ritz_resid_max": float(np.max(resid)),
                 "setup_wave_solves": 1024}
    else:
        g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
        setup = {"basis": "closed-form sine vectors"}
    if args.compress > 0.0 and w.dim == 2:
        try:
            ranks = g.whv_compress_basis(args.compress)
            ny, nx = w.npts[1] - 2, w.npts[0] - 2
            setup.update({"compressed_tau": args.compress, "compressed_rank_mean": float(np.mean(ranks)),
                          "compressed_rank_max": int(max(ranks)),
                          "compression_ratio": float(sum(r * (nx + ny + 1) for r in ranks) / (len(ranks) * nx * ny))})
        except whv.WhvError as e:   # not compressible at this tolerance: the basis stays dense
            setup.update({"compressed_tau": args.compress, "compression": f"refused: {e}"})
    if cons:
        setup["operator"] = "conservative div(c^2 grad), second order, Euclidean inner products"
    setup["setup_s"] = time.perf_counter() - t0
    if args.steps_per_sweep:
        g.whv_set_steps_per_sweep(args.steps_per_sweep)
        setup["steps_per_sweep"] = args.steps_per_sweep
    elif w.dim >= 2:
        setup["steps_per_sweep"] = g.whv_autotune(prm)   # 2-D: blocked k; 3-D: one or two steps per launch
    f = dev(I.forcing_for(w))
    u = torch.zeros_like(f)
    res = {}

    def step():
        res["info"] = g.whv_solve(prm, f, u)[1]
    ms, _ = _timed(stream, step, args.steps, args.warmup, flush if w.n_unknowns < 30_000_000 else None)
    info = res["info"]
    prm_chk = whv.make_params(w.omega, method=method, tol=w.tol, maxit=20000, restart=30, true_residual=True,
                              refine_fp64=refine)
    _, ichk = g.whv_solve(prm_chk, f, u)
    lups = info["wave_solves"] * info["nt"] * w.n_unknowns
    line.update({"workload": name, "value": ms, "ms_per_step": ms,
                 "dtype": "f64" if prec == whv.WHV_FP64 else "f32", "krylov_dtype": "f64",
                 "config": dict({"workload": name, "grid": list(w.npts), "order": order, "omega": w.omega,
                                 "nd": w.nd, "tol": w.tol, "method": method.upper(),
                                 "variable_speed": bool(w.speed), "nt": info["nt"],
                                 "correction_residuals": ("df64" if dfres else "fp64") if refine else None},
                            **setup),
                 "iterations": info["iterations"], "outer_iterations": info["outer_iterations"],
                 "wave_solves": info["wave_solves"], "glups_solve": lups / (ms * 1e-3) / 1e9,
                 "accuracy": {"true_rel_residual": ichk["true_rel_residual"]}})
    if name == "c3":
        # break-even of the eigenvector set-up (Sec. 4.1 cost model): the same problem without
        # deflation, counted in wave solves, outside the timed region
        g0 = whv.Grid(w.npts, order=order, precision=prec, stream=stream)
        if w.speed:
            if cons:
                g0.whv_set_speed_form(dev(I.speed_squared(w.speed, w.npts, w.speed_seed)), whv.WHV_SPEED_CONSERVATIVE)
            else:
                g0.whv_set_speed(dev(I.speed_squared(w.speed, w.npts, w.speed_seed)))
        p0 = whv.make_params(w.omega, method="cg", tol=w.tol, maxit=20000, refine_fp64=refine)
        t0 = time.perf_counter()
        _, i0 = g0.whv_solve(p0, f)
        t_undefl = time.perf_counter() - t0
        setup_ws = setup["setup_wave_solves"] + w.nd   # eigen-solve + A W of Algorithm 4 (first solve)
        gain = i0["wave_solves"] - info["wave_solves"]
        line["break_even"] = {"setup_wave_solves": setup_ws, "wave_solves_deflated": info["wave_solves"],
                              "wave_solves_undeflated": i0["wave_solves"], "undeflated_status": i0["status"],
                              "undeflated_s": t_undefl,
                              "rhs": (setup_ws / gain) if gain > 0 else None}
        g0.close()
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    args = parse(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch_under_torchrun(args, argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c4":
        return run_c4(args)
    if args.workload == "c4wave":
        return run_c4wave(args)
    if args.workload == "stencil3d":
        return run_stencil3d(args)
    if args.workload == "c2":
        return run_c2(args)
    return run_workload(args)


if __name__ == "__main__":
    sys.exit(main())
