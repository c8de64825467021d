#!/usr/bin/env python
"""Benchmark of the deflated WaveHoltz solve on one B300 (replicas on N GPUs).

A step is one complete deflated solve of the 2-D Helmholtz workload: 513^2 nodes (511^2
unknowns), omega = 50, Gaussian source of width 0.02 at a seeded point, 64 closed-form sine
eigenvectors (DEVD, Algorithm 2) and CG on (I - S_h) u = b to relative residual 1e-6 -- weight
tables, Taylor start, the fused leapfrog + filter steps, the operator epilogue, forcing deflation
and inflation and the FP64 Krylov reductions all run in the library's kernels.  Default precision:
FP32 wave stepping with FP64 Krylov / deflation arithmetic; --precision fp64 runs the plain FP64
form (tolerance 1e-8, the 2-D workload's own).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64] [--impl whv|reference]

Prints one JSON line on rank 0.  --impl reference times the FP64 CPU oracle (numpy, one thread)
on the same workload instead.  Under torchrun every rank solves its own copy of the workload
(replicas; the path has no collective) and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import re
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
# the CPU oracle legs run single-threaded (numpy elementwise work is single-threaded anyway;
# this pins the BLAS calls of the projections too); set before numpy is first imported
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

METRIC = "WaveHoltz solve time to rel. residual 1e-6; stencil GLUP/s vs HBM roofline"
L2_FLUSH_BYTES = 512 << 20   # > 126 MB L2: written between timed steps


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="whv", choices=["whv", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--method", default="", choices=["", "cg", "dcg", "gmres", "agmres", "abicgstab"],
                    help="accelerator of the single-grid workloads (default: DCG for c1/c3, CG otherwise)")
    ap.add_argument("--steps-per-sweep", type=int, default=0,
                    help="2-D stepping kernel: 0 = autotune (default), k = blocked k steps per launch, "
                         "-k = persistent kernel; a fixed value keeps profiled runs on the kernel the plain run uses")
    ap.add_argument("--residual", default="df64", choices=["df64", "fp64"],
                    help="FP32 stepping: precision of the b and residual wave solves of the correction "
                         "(df64 = pairs of FP32 with error-free arithmetic; the accuracy check always uses FP64)")
    ap.add_argument("--check-every", type=int, default=1,
                    help="convergence test every k iterations; 1 keeps the CG loop on the device (a graph "
                         "with a conditional node), k > 1 launches one iteration graph per step from the host")
    ap.add_argument("--eigs", default="lanczos", choices=["lanczos", "thick"],
                    help="variable-speed workload: one 1024-step Lanczos run, or thick-restart Lanczos (basis 3 nd + 4)")
    ap.add_argument("--compress", type=float, default=0.0,
                    help="variable-speed workload: SVD-compress the basis with this Frobenius tolerance")
    ap.add_argument("--form", default="nonconservative", choices=["nonconservative", "conservative"],
                    help="variable-speed workload: operator form (conservative: div(c^2 grad), second order)")
    ap.add_argument("--sources", type=int, default=0,
                    help="batched workload: Gaussian sources per (grid, frequency) (default 16)")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "study"],
                    help="c2 (default): the 513^2 deflated solve; others: the 1-D, variable-speed "
                         "1025^2, batched and 3-D workloads, measured on request")
    return ap.parse_args()


def workload_config(precision):
    from paper_2606_31842_b300 import inputs as I
    w = I.WORKLOADS["c2"]
    tol = 1e-6 if precision == "fp32" else w.tol
    return w, tol


def config_dict(w, tol, precision, nt, n_gpus):
    return {"workload": f"2-D Helmholtz {w.npts[0]}x{w.npts[1]} nodes, omega={w.omega:g}, Gaussian source width 0.02, "
                        f"DEVD + CG with {w.nd} closed-form eigenvectors, tol {tol:g}",
            "grid": list(w.npts), "unknowns": w.n_unknowns, "omega": w.omega, "nd": w.nd, "tol": tol,
            "method": "DEVD-CG" + (" in FP64 residual correction" if precision == "fp32" else ""),
            "stepping": precision, "krylov": "fp64", "nt": nt,
            "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{n_gpus}"}


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
def oracle_sample(w, tol, iterations_hint, budget_s=12.0):
    """Time the FP64 oracle on a bounded sample of the workload: mode selection + basis, b, and
    as many CG iterations as fit in the budget; extrapolate to `iterations_hint` iterations."""
    from oracle import operators as O, waveholtz as WH, spectral as SP, krylov as K
    from paper_2606_31842_b300 import inputs as I
    g = O.Grid(w.npts)
    tg = WH.time_grid_for(g, w.omega)
    f = I.forcing_for(w)
    t0 = time.perf_counter()
    modes, lam2, _ = SP.select_modes(g, tg, w.nd)
    V = SP.basis(g, modes)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = WH.rhs_b(g, tg, K.project_out(g, V, f))
    t_b = time.perf_counter() - t0
    A = K.Operator(g, tg)
    k = max(1, int(budget_s / max(t_b, 1e-3)))
    t0 = time.perf_counter()
    K.cg(g, A, b, 0.0, k)
    t_it = (time.perf_counter() - t0) / k
    solve_s = t_b + iterations_hint * t_it
    return {"solve_s": solve_s, "setup_s": t_setup, "t_wave": t_b, "t_iter": t_it, "k": k}


def run_reference(args):
    """--impl reference: the FP64 CPU oracle on the same workload, metric and unit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, tol = workload_config(args.precision)
    from oracle import operators as O, waveholtz as WH
    nt = WH.time_grid_for(O.Grid(w.npts), w.omega).nt
    # iteration count of the oracle at this tolerance (deflated CG on this workload)
    iters = 37 if tol >= 1e-6 else 50
    times = []
    for s in range(args.warmup + args.steps):
        t = oracle_sample(w, tol, iters, budget_s=3.0)
        if s >= args.warmup:
            times.append(t["solve_s"] * 1e3)
    ms = statistics.mean(times)
    cb = {"value": ms, "unit": "ms", "cores": 1, "kind": "oracle",
          "sample": f"b wave solve + {t['k']} CG iterations per step at 1 thread, extrapolated to {iters} iterations"}
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(w, tol, "fp64", nt, args.gpus), "cpu_baseline": cb,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------ GPU arm
# the sources a recorded traffic figure depends on: whole files, or (file, kernel) for the text of
# one kernel's definition in a file that holds others as well
KERNEL_SOURCES = {
    "k_block2d": ("stencil_blocked.cu", "quad2d.cuh", "whv_device.cuh"),
    "k_step3d": (("stencil.cu", "k_step3d"), "stencil_ops.cuh", "whv_device.cuh"),
    "k_step3d2": (("stencil.cu", "k_step3d2"), "stencil_ops.cuh", "whv_device.cuh"),
}


def _kernel_text(src, name):
    """The definition of __global__ kernel `name` in `src`: from its declaration to the closing
    brace of its body."""
    m = re.search(r"__global__[^;{]*?\b" + re.escape(name) + r"\(", src)
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


def run_workload(args):
    """The other workloads (one JSON line each): 1-D FP64 DCG, variable-speed 1025^2 with the device
    Lanczos basis, the batched squares and the 3-D cube."""
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
    if args.workload == "c4":
        # FP32 stepping inside FP64 residual correction (default), or the plain FP64 form
        fp32 = args.precision == "fp32"
        gprec = whv.WHV_FP32_STEP if fp32 else whv.WHV_FP64
        probs = []
        t0 = time.perf_counter()
        nsrc = args.sources if args.sources > 0 else I.C4_SOURCES
        for n in I.C4_SIZES:
            for om in I.C4_OMEGAS:
                w = I.WORKLOADS[f"c4_{n}_{int(om)}"]
                prm = whv.make_params(om, method="cg", tol=w.tol, maxit=3000, refine_fp64=fp32,
                                      residual_df64=fp32 and args.residual == "df64", check_every=args.check_every)
                tmpl = whv.Grid(w.npts, precision=gprec, stream=stream)
                tmpl.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
                b = tmpl.whv_get_basis(want_vectors=True)
                for src in range(nsrc):
                    g = whv.Grid(w.npts, precision=gprec, stream=stream)
                    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_USER, V=b["V"].reshape(-1),
                                              lambda2=b["lambda2"], flags=whv.WHV_BASIS_EXACT)
                    probs.append((g, prm, dev(I.forcing_for(w, src)), w))
                tmpl.close()
        setup_s = time.perf_counter() - t0
        grids = [p[0] for p in probs]
        params = [p[1] for p in probs]
        if args.steps_per_sweep > 0:
            grids[0].whv_set_steps_per_sweep(args.steps_per_sweep)
            kb, ktag = args.steps_per_sweep, "fixed"
        else:
            kb, ktag = whv.whv_autotune_batched(grids, params), "autotuned"   # batched kernel's k
        fs = [p[2] for p in probs]
        us = [torch.zeros(g.N, dtype=torch.float64, device="cuda") for g in grids]
        res = {}

        def step():
            _, infos = whv.whv_solve_batched(grids, params, fs, us)
            res["infos"] = infos
        ms, _ = _timed(stream, step, args.steps, args.warmup, None)
        infos = res["infos"]
        lups = sum(g.N * i["nt"] * i["wave_solves"] for g, i in zip(grids, infos))
        lups64 = sum(g.N * i["nt"] * i["wave_solves_fp64"] for g, i in zip(grids, infos))
        # FP64 true residual of a sample of the problems, recomputed on separate FP64 grids
        # (outside the timed region)
        chk = []
        for k in range(0, len(probs), 37):
            g, prm, f, w = probs[k]
            g64 = whv.Grid(w.npts, precision=whv.WHV_FP64, stream=stream)
            r = g64.whv_apply_pi(prm, us[k], f)
            b = g64.whv_apply_pi(prm, torch.zeros_like(f), f)
            chk.append(float((r - us[k]).norm() / b.norm()))
            g64.close()
        form = (("DEVD-CG with FP32 stepping inside FP64 residual correction"
                 + (" (double-float b and residual wave solves)" if args.residual == "df64" else ""))
                if fp32 else "DEVD-CG, FP64 stepping")
        line.update({"workload": "c4", "value": ms, "ms_per_step": ms, "dtype": "f32" if fp32 else "f64",
                     "krylov_dtype": "f64",
                     "config": {"workload": f"batched: 4 squares (257..1025)^2 x 4 omega x {nsrc} Gaussian sources "
                                            f"(width 2h), 32 closed-form vectors each, {form} to 1e-6; every "
                                            f"batched wave solve of all {len(probs)} problems is one persistent launch",
                                "problems": len(probs), "setup_s": setup_s,
                                "steps_per_sweep": f"{kb} ({ktag}, both precisions)",
                                "check_every": args.check_every},
                     "iterations_max": max(i["iterations"] for i in infos),
                     "iterations_mean": statistics.mean(i["iterations"] for i in infos),
                     "outer_iterations_max": max(i["outer_iterations"] for i in infos),
                     "wave_solves_fp64": sum(i["wave_solves_fp64"] for i in infos),
                     "wave_solves": sum(i["wave_solves"] for i in infos),
                     "glups_solve": lups / (ms * 1e-3) / 1e9, "glups_fp64_share": lups64 / max(lups, 1),
                     "accuracy": {"fp64_true_rel_residual_max": (max(i["true_rel_residual"] for i in infos) if fp32
                                                                   else None),
                                  "fp64_true_rel_residual_recomputed_sample_max": max(chk)}})
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
                                                   fp64_stepping=False)
        setup = {"basis": f"device thick-restart Lanczos on S_h (FP32 stepping, basis {3 * w.nd + 4}, tol 1e-6)",
                 "ritz_resid_median": float(np.median(resid)), "ritz_resid_max": float(np.max(resid)),
                 "setup_wave_solves": st["wave_solves"], "restarts": st["restarts"], "converged": st["converged"]}
    elif name == "c3":
        theta, resid = g.whv_lanczos(prm, w.nd, 1024, None, False, 0)
        setup = {"basis": "device Lanczos on S_h (FP32 stepping, 1024 steps)",
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


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        return run_workload(args)
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2606_31842_b300 import build as whv_build
    whv_build.build()
    from paper_2606_31842_b300 import whv
    from paper_2606_31842_b300 import inputs as I

    w, tol = workload_config(args.precision)
    prec = whv.WHV_FP32_STEP if args.precision == "fp32" else whv.WHV_FP64
    stream = torch.cuda.Stream()
    g = whv.Grid(w.npts, precision=prec, stream=stream)
    # FP32 stepping runs inside FP64 residual correction so that the FP64 residual meets tol
    fp32 = args.precision == "fp32"
    prm = whv.make_params(w.omega, method="cg", tol=tol, maxit=5000, check_every=args.check_every,
                          refine_fp64=fp32, residual_df64=fp32 and args.residual == "df64")
    tgrid = g.whv_time_grid(prm)
    nt = tgrid["nt"]
    g.whv_set_deflation_basis(prm, w.nd, whv.WHV_BASIS_CLOSED_FORM)
    if args.steps_per_sweep:
        g.whv_set_steps_per_sweep(args.steps_per_sweep)
        ksweep = args.steps_per_sweep
    else:
        ksweep = g.whv_autotune(prm)                  # steps per sweep of the blocked 2-D kernel
    f_host = torch.from_numpy(I.forcing_for(w).ravel()).pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    with torch.cuda.stream(stream):
        f = f_host.to("cuda", non_blocking=True)
        u = torch.zeros_like(f)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream.synchronize()

    def solve():
        return g.whv_solve(prm, f, u)[1]

    for _ in range(max(3, args.warmup)):
        info = solve()
    # ------------------------------------------------------------------ timed region
    times, infos = [], []
    launches0 = whv.whv_kernel_launches()
    with ClockSampler(local) as clk:
        time.sleep(0.5)                               # let the sampler start
        barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")           # lets a profiler restrict itself to these steps
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)                      # evict the working set from L2
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(solve())
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        barrier()
    launches = whv.whv_kernel_launches() - launches0
    clocks = clk.summary()
    ms = aggregate_max(statistics.mean(times), world, device="cuda")
    info = infos[-1]
    lups = info["wave_solves"] * nt * w.n_unknowns
    # accuracy of the timed configuration (outside the timed region): FP64 true residual and
    # the error against an FP64-stepping solve of the same problem on the same GPU
    prm_chk = whv.make_params(w.omega, method="cg", tol=tol, maxit=5000, true_residual=True,
                              refine_fp64=fp32, residual_df64=fp32 and args.residual == "df64")
    u_chk, info_chk = g.whv_solve(prm_chk, f)
    accuracy = {"true_rel_residual": info_chk["true_rel_residual"],
                "true_residual_check": "FP64 wave solves",
                "correction_residuals": ("fp64" if not fp32 else
                                         "df64 (pairs of FP32)" if args.residual == "df64" else "fp64")}
    if args.precision == "fp32":
        g64 = whv.Grid(w.npts, precision=whv.WHV_FP64, stream=stream)
        prm64 = whv.make_params(w.omega, method="cg", tol=1e-11, maxit=5000)
        g64.whv_set_deflation_basis(prm64, w.nd, whv.WHV_BASIS_CLOSED_FORM)
        u64, _ = g64.whv_solve(prm64, f)
        accuracy["rel_max_err_vs_fp64_solve"] = float((u_chk - u64).abs().max() / u64.abs().max())
        g64.close()
    glups_solve = lups / (ms * 1e-3) / 1e9

    # ------------------------------------------------------------------ e2e: host buffers
    e2e_times = []
    for k in range(args.steps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0.record(stream)
            f.copy_(f_host, non_blocking=True)
        g.whv_solve(prm, f, u)
        with torch.cuda.stream(stream):
            u_host.copy_(u, non_blocking=True)
            e1.record(stream)
        e1.synchronize()
        if k > 0:
            e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = statistics.mean(e2e_times)

    # ------------------------------------------------------------------ dominant kernel
    # the leapfrog+filter kernel of the timed solve's wave solves -- k_block2d (k steps per launch)
    # when the autotuner picked k > 1, else k_step: average time per leapfrog step over replays of
    # the same wave-solve graph, timed with events on the launching stream right after the timed
    # region; algorithmic bytes = 5 s per LUP (read W^n, W^{n-1}, acc; write W^{n+1}, acc) times
    # the k N LUPs one launch advances
    reps = 20
    v = torch.randn(w.n_unknowns, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    torch.cuda.synchronize()
    g.whv_apply_pi(prm, v, None, out)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        g.whv_apply_pi(prm, v, None, out)
    e1.record(stream)
    e1.synchronize()
    t_step = e0.elapsed_time(e1) * 1e-3 / (reps * nt)
    esz = 4 if args.precision == "fp32" else 8
    bytes_per_lup = 5 * esz                          # read W^n, W^{n-1}, acc; write W^{n+1}, acc
    achieved = bytes_per_lup * w.n_unknowns / t_step / 1e9
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs", 6400.0)
    kname = "k_block2d" if ksweep > 1 else "k_step"
    kdesc = (f"k_block2d ({ksweep} fused leapfrog steps + trapezoid filter per launch)" if ksweep > 1
             else "k_step (fused leapfrog step + trapezoid filter)")
    traffic = traffic_for(kname, args.precision)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kdesc,
            "bytes_per_lup": bytes_per_lup, "lups_per_launch": w.n_unknowns * max(1, ksweep),
            "launch_us": t_step * max(1, ksweep) * 1e6, "step_us": t_step * 1e6,
            "glups": w.n_unknowns / t_step / 1e9,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "note": "the 511^2 state (3 arrays, 3 MB) stays resident in the 126 MB L2 during a wave solve"}

    # ------------------------------------------------------------------ HBM-bound stencil
    # the 3-D 256^3 grid (66 MB per FP32 array, 3 arrays > L2): f = 0 wave solves of the
    # 7-point z-marching step kernel, the case on which the HBM fraction is meaningful
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
        # per step: the first-step kernel's share is 1/nt of the launches; the wave-solve mean
        return e0.elapsed_time(e1) * 1e-3 / (reps3 * nt3)

    t31 = time_3d(1)    # k_step3d, one step per launch
    t32 = time_3d(2)    # k_step3d2, two steps per launch
    ach31, ach32 = 20 * g3.N / t31 / 1e9, 20 * g3.N / t32 / 1e9
    stencil_hbm = {"kernel": "k_step3d2 (3-D 7-point, two leapfrog steps + filter per launch, FP32)",
                   "workload": "256^3 nodes (254^3 unknowns), omega=40, f = 0 wave solves, nt=%d" % nt3,
                   "bound": "hbm", "achieved": ach32, "peak": peak, "unit": "GB/s", "frac": ach32 / peak,
                   "bytes_per_lup": 20, "glups": g3.N / t32 / 1e9, "step_us": t32 * 1e6,
                   "own_bytes_per_lup": 12, "own_frac": 12 * g3.N / t32 / 1e9 / peak,
                   "traffic": traffic_for("k_step3d2", "fp32"), "traffic_unit": "DRAM bytes per launch (2 steps)",
                   "note": "achieved/frac count the 20 B per LUP of single-step streaming (equivalent "
                           "bandwidth); own_frac counts the 12 B per LUP the two-step kernel must move",
                   "single_step": {"kernel": "k_step3d (one step per launch)", "achieved": ach31,
                                   "frac": ach31 / peak, "glups": g3.N / t31 / 1e9, "step_us": t31 * 1e6,
                                   "traffic": traffic_for("k_step3d", "fp32")}}
    g3.close()
    del v3, o3

    line = {"metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "krylov_dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(w, tol, args.precision, nt, world), steps_per_sweep=ksweep,
                           check_every=args.check_every,
                           correction_residuals=("df64" if fp32 and args.residual == "df64" else "fp64")),
            "iterations": info["iterations"], "wave_solves": info["wave_solves"],
            "rel_residual": info["rel_residual"], "glups_solve": glups_solve, "accuracy": accuracy,
            "outer_iterations": info.get("outer_iterations", 0), "wave_solves_fp64": info.get("wave_solves_fp64", 0),
            "roofline": roof, "stencil_hbm": stencil_hbm,
            "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": w.n_unknowns * 8,
                    "d2h_bytes_per_step": w.n_unknowns * 8},
            "gpu_launches": launches, "clocks": clocks}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = oracle_sample(w, tol, info["iterations"])
        line["cpu_baseline"] = {"value": cb["solve_s"] * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                                "sample": f"oracle (numpy FP64, 1 thread): b wave solve + {cb['k']} CG iterations, "
                                          f"extrapolated to the GPU's {info['iterations']} iterations"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
