#!/usr/bin/env python
"""Benchmark of the posterior-mean solve on one GB300 (or N independent ranks).

One step = one solve of G X = B (eq. mu*) to true FP64 relative residual 1e-8 with the
mixed-precision path (FP32 preconditioned CG inside FP64 iterative refinement), on the
1024 x 2048 latitude-longitude sphere workload (n = 2,097,152 pixels, k = 6 sources, m = 9
Planck channels), with B resident in HBM.  Reported beside it: the same solve in plain FP64
PCG, the stand-alone operator apply in GB/s, the roofline of the dominant kernel, an
end-to-end number through the public API with host buffers, and the CPU oracle timed on a
bounded sample.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead.
"""

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solve time to relres 1e-8 (mixed vs FP64 CG, 1 GB300); operator HBM GB/s"
WORKLOAD = "sphere1024x2048_k6_m9"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--scale", type=int, default=1, help="divide grid sides (small runs)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--pixel-order", default="row", choices=["row", "blocked"],
                    help="pixel numbering of the main workload: row-major image, or 16 x 16 "
                         "blocks (most stencil neighbours in a pixel's own 256-pixel tile)")
    ap.add_argument("--profile-case", action="store_true",
                    help="one untimed solve and three applies of the workload (for ncu)")
    ap.add_argument("--paper-model", action="store_true",
                    help="the paper's own model on the workload grid: printed physical mixing "
                         "and channel weights (App. B), intrinsic GMRF prior (App. C)")
    ap.add_argument("--learn", type=int, default=0, metavar="N",
                    help="N steps of parameter learning on the 512 x 1024 workload, warm and cold")
    ap.add_argument("--variance", type=int, default=0, metavar="S",
                    help="posterior variances of the workload from S Rademacher probes")
    ap.add_argument("--variance-probing", type=int, default=0, metavar="P",
                    help="posterior variances of the workload by probing with a distance-(P-1) "
                         "colouring (P^2 k probes), with the change against P/2 as the error "
                         "estimate")
    ap.add_argument("--separable", action="store_true",
                    help="separable special case of the workload: block-Lanczos Sylvester "
                         "solver (Algorithms 4 and 5) against the preconditioned CG")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# algorithmic bytes per pixel: every stream a kernel must read or write once per pixel
# ---------------------------------------------------------------------------------------------
def bytes_inner_apply(k, m, E, s=4):
    # read z, p, q, d (4k) + D (m) + ELL values (E) + diagonal (1); write p, q, d (3k); ELL
    # cols int32 (the previous iteration's d += alpha p is done here, where p is read anyway)
    return (7 * k + m + E + 1) * s + 4 * E


def bytes_inner_update(k, m, s=4):
    # read r, q (2k) + preconditioner scaling (k, FP32) + factor (k(k+1)/2, FP16);
    # write r, z (2k)
    return (5 * k) * s + 2 * (k * (k + 1) // 2)


def fp64_ops_inner(k, E):
    """FP64 floating-point operations per pixel of one FP64 PCG iteration (an FMA is two), as
    the FP64 kernels compute them: the operator kernel (pixel block k^2 FMAs, stencil E k, the
    tau scaling k, d, p and q updates 3k, p . q k) and the update kernel (r update k, block
    solve k(k-1) FMAs and 4k multiplies, r . z and r . r 2k)."""
    apply_fma = k * k + E * k + 5 * k
    update_fma, update_mul = k * k + 2 * k, 4 * k
    return 2 * apply_fma + 2 * update_fma + update_mul


def bytes_inner_fp64(k, E):
    """Bytes per pixel of one FP64 PCG iteration: operator kernel reads z, p, q, d, the FP64
    pixel block (k(k+1)/2), ELL values (FP64) and columns, writes p, q, d; update kernel reads
    r, q and the FP64 factor (k + k(k+1)/2), writes r, z."""
    nb = k * (k + 1) // 2
    return (7 * k * 8 + nb * 8 + E * 8 + 4 * E) + (4 * k * 8 + (k + nb) * 8)


def fp64_peak_tflops(dev):
    """Measured FP64 peak of this GPU: a cuBLAS DGEMM of 4096^3 (2 n^3 operations) through
    torch, best of 5 timed with CUDA events after 2 warm-ups (the dense FP64 rate this part
    reaches; the FP64 PCG kernels do FMAs and multiplies on the same units)."""
    import torch
    n = 4096
    g = torch.Generator(device=dev).manual_seed(0)
    a = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    b = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    for _ in range(2):
        torch.matmul(a, b)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def bytes_apply(k, m, E, R=1, s=4):
    # read X (R k) + D (m) + ELL values (E) + diagonal (1); write Y (R k); ELL cols int32
    return (2 * R * k + m + E + 1) * s + 4 * E


def kernel_name(kind, variant, k, m, E):
    """Name of the inner kernel a solve ran (variant as reported in sylv_info)."""
    shape = f"{k},{m},{E}" if E else f"{k},0,0"
    if kind == "apply":
        return {0: f"k_inner_apply<{shape},float>", 1: f"k_inner_apply_tma<{shape}>",
                2: f"k_inner_apply_mc<{shape}>"}[variant]
    return {0: f"k_inner_update<{shape},float>", 1: f"k_inner_update_tma<{k},{m}>",
            2: f"k_inner_update_mc<{k},{m}>"}[variant]


KERNEL_SOURCES = ["pcg_kernels.cuh", "pcg_tma.cuh", "sylv_internal.cuh"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2204_08057_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch of ``kernel`` recorded in profiles/ by an ncu capture, if the
    kernel sources are unchanged since (else None)."""
    import glob
    import re
    cur = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        m = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]{16})", text)
        if not m or m.group(1) != cur:
            continue
        m = re.search(r"traffic_bytes_per_launch\[" + re.escape(kernel) + r"\]:\s*([0-9.eE+]+)",
                      text)
        if m:
            return float(m.group(1))
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------------------------
def oracle_pcg_sample(p, seconds, iters_ref):
    """Times the oracle's block-Jacobi PCG (FP64, numpy/scipy) on the full workload for a
    bounded number of iterations; scales ms/iteration to a whole solve of ``iters_ref``
    iterations.  Returns a cpu_baseline dict."""
    from oracle import model, solve
    L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
    A = model.powerlaw_mixing(p.nu, p.beta)
    b = model.rhs(p.D, p.Yobs[0], A)
    t0 = time.perf_counter()
    _, it, _, secs = solve.pcg_block_jacobi(L, p.D, p.tau, p.kappa, A, b, eps=1e-8,
                                            maxit=10 ** 9, max_seconds=seconds)
    wall = time.perf_counter() - t0
    per_it = secs / max(it, 1)
    return {
        "value": per_it * iters_ref * 1e3, "unit": "ms", "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": (f"oracle FP64 block-Jacobi PCG (numpy/scipy, default threading) on the full "
                   f"{p.name} system: {it} iterations in {secs:.1f} s ({wall:.1f} s with set-up); "
                   f"ms/iteration x {iters_ref} iterations (the FP64 PCG iteration count to "
                   f"relres 1e-8)"),
        "ms_per_iteration": per_it * 1e3, "iterations_timed": it,
    }


def oracle_pcg_full(p):
    """Times one whole solve of the oracle's block-Jacobi PCG (FP64, numpy/scipy) on the full
    workload to recursive relres 1e-8, and reports its true FP64 relres.  Returns a
    cpu_baseline dict (a measured solve, no projection)."""
    from oracle import model, solve
    L = model.laplacian_from_csr(p.graph.rowptr, p.graph.col, p.graph.val, p.n)
    A = model.powerlaw_mixing(p.nu, p.beta)
    b = model.rhs(p.D, p.Yobs[0], A)
    t0 = time.perf_counter()
    x, it, rel_rec, secs = solve.pcg_block_jacobi(L, p.D, p.tau, p.kappa, A, b, eps=1e-8)
    wall = time.perf_counter() - t0
    rel_true = solve.relres(L, p.D, p.tau, p.kappa, A, x, b)
    return {
        "value": secs * 1e3, "unit": "ms", "cores": os.cpu_count(), "kind": "oracle",
        "sample": (f"one whole solve of the oracle's FP64 block-Jacobi PCG (numpy/scipy, default "
                   f"threading) on the full {p.name} system to relres 1e-8: {it} iterations in "
                   f"{secs:.1f} s ({wall:.1f} s with set-up), true relres {rel_true:.2e}"),
        "measured": "whole solve", "iterations": it, "relres_true": rel_true,
    }


def stored_iterations(config):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_pcg_iterations_c{config}.json")
    try:
        with open(path) as f:
            return int(json.load(f)["iterations"])
    except Exception:
        return None


# ---------------------------------------------------------------------------------------------
def run_reference(args, rank, world):
    import synth
    if rank != 0:
        return
    p = synth.config_problem(args.config, scale=args.scale)
    iters = stored_iterations(args.config)
    vals = []
    walls = []
    sample = None
    # a step is one bounded sample of the solve (the whole run stays within a few minutes);
    # the value is the sample's ms per iteration times the oracle's iteration count to 1e-8
    per_step = max(3.0, min(args.cpu_seconds, 150.0 / max(args.steps + args.warmup, 1)))
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = oracle_pcg_sample(p, per_step, iters or 1)
        if step >= args.warmup:
            walls.append(time.perf_counter() - t0)
            vals.append(cb["value"])
            sample = cb
    v = float(np.mean(vals))
    if iters is None:
        sample["sample"] += " [no stored oracle iteration count: value is ms per iteration]"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "precision": "FP64 (the CPU oracle)",
            "value_is": "projection: ms per oracle iteration (timed) x the oracle's iteration "
                        "count to relres 1e-8; ms_per_step is the wall time of one bounded "
                        "sample step",
            "config": main_config(p),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": sample["cores"],
                             "kind": "oracle", "sample": sample["sample"]},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main_config(p):
    """The `config` of the main workload's line (both arms print the same)."""
    return {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "nrhs": 1, "tol": 1e-8,
            "l2": "inputs larger than L2 (working set ~%d MB)"
                  % int((p.n * (5 * p.k * 4 + 2 * p.k * 8 + p.m * 12 + 44)) / 1e6),
            "per_rank": "independent instance per rank (own seed)"}


def with_order(p, order):
    """The problem in the requested pixel numbering (the solution is the same, renumbered)."""
    if order == "row":
        return p
    import synth
    return synth.permute_problem(p, synth.blocked_order(p.graph.H, p.graph.W, 16, 16))


def rank_problem(config, rank, scale=None, order="row"):
    """Weak scaling: rank r solves its own instance of the workload (same grid and shape,
    its own seeded noise maps, spectral parameters and observations)."""
    import synth
    p = synth.config_problem(config, scale=scale)
    if rank > 0:
        p = synth.make_problem(p.name, p.graph, p.k, p.nu, None, None, p.tau,
                               synth.CONFIG_SEED_BASE + 100 * rank + config,
                               beta_draw=(-3.0, 2.0), kappa_draw=(0.01, 1.0), tol=p.tol,
                               nrhs=p.nrhs) if config in (2, 4, 5) else \
            synth.make_problem(p.name, p.graph, p.k, p.nu, p.beta, p.kappa, p.tau,
                               synth.CONFIG_SEED_BASE + 100 * rank + config, tol=p.tol,
                               nrhs=p.nrhs)
    return with_order(p, order)


def max_over_ranks(value, dist, device="cpu"):
    """The slowest rank's time (every rank gets it)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, local_rank):
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    from paper_2204_08057_gb300.operator import Operator

    _build.build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

    # weak scaling: every rank solves its own independent instance (own seed)
    p = rank_problem(args.config, rank, args.scale, args.pixel_order)
    # set-up (sylv_create: CSR check, sliced ELL, copies of D, FP64 pixel blocks and factors)
    Op0 = Operator(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=p.D, tau=p.tau,
                   kappa=p.kappa, nu=p.nu, beta=p.beta)
    Op0.close()
    rp = torch.as_tensor(p.graph.rowptr, device=dev)
    cl = torch.as_tensor(p.graph.col, device=dev)
    vl = torch.as_tensor(p.graph.val, device=dev)
    Dd = torch.as_tensor(p.D, device=dev)
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    op = Operator(rowptr=rp, col=cl, val=vl, D=Dd, tau=p.tau, kappa=p.kappa, nu=p.nu,
                  beta=p.beta)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t_setup) * 1e3
    E = int(np.max(np.diff(p.graph.rowptr))) - 1
    Yh = torch.from_numpy(p.Yobs).pin_memory()
    Y = Yh.to(dev)
    B = op.rhs(Y)
    stream = torch.cuda.current_stream()
    ms_rhs, _ = _timed(stream, lambda: op.rhs(Y), 10)
    rhs_bytes = (p.m * 8 + p.m * 8 + p.k * 8) * p.n      # Y, D (FP64) in, B out

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- mixed-precision solve (the step) ------------------------------------------------------
    # timed without per-kernel events (an event pair around every launch inside the captured
    # graphs costs ~8 % of the solve); the kernel breakdown comes from a profiled pass below
    kw = dict(tol=1e-8, precision=1, profile=0)
    for _ in range(args.warmup):
        X, info = op.solve(B, **kw)
    clocks = ClockSampler(local_rank) if not args.no_clocks else None
    barrier()
    if clocks:
        clocks.start()
        time.sleep(0.5)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for _ in range(args.steps):
        X, info = op.solve(B, **kw)
        infos.append(info)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop() if clocks else {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
    ms = max_over_ranks(ms, dist, dev)
    assert infos[-1]["code"] == 0, infos[-1]
    launches_timed = int(sum(i["launches"] for i in infos))

    # ---- profiled pass: the same solves with CUDA events around every kernel launch --------
    kwp = dict(tol=1e-8, precision=1, profile=1)
    infos = []
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    p0.record(stream)
    for _ in range(args.steps):
        X, info = op.solve(B, **kwp)
        infos.append(info)
    p1.record(stream)
    barrier()
    ms_profiled = p0.elapsed_time(p1) / args.steps
    last = infos[-1]
    assert last["code"] == 0, last

    # ---- plain FP64 PCG on the same system ----------------------------------------------------
    # timed without per-kernel events like the mixed solve; then one profiled solve gives its
    # kernel times for the FP64 roofline
    kw64 = dict(tol=1e-8, precision=0, profile=0)
    X64, info64 = op.solve(B, **kw64)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    f0.record(stream)
    for _ in range(args.fp64_steps):
        X64, info64 = op.solve(B, **kw64)
    f1.record(stream)
    barrier()
    ms64 = f0.elapsed_time(f1) / max(args.fp64_steps, 1)
    _, info64p = op.solve(B, tol=1e-8, precision=0, profile=1)
    relerr_mixed_vs_fp64 = float(torch.linalg.norm(X - X64) / torch.linalg.norm(X64))
    peak64 = fp64_peak_tflops(dev)
    its64 = max(info64p["iterations"], 1)
    ms_it64 = (info64p["ms_apply"] + info64p["ms_update"]) / its64
    flops64 = fp64_ops_inner(p.k, E) * p.n
    bytes64 = bytes_inner_fp64(p.k, E) * p.n
    fp64_roof = {
        "bound": "fp64",
        "achieved_tflops": flops64 / (ms_it64 * 1e-3) / 1e12, "peak_tflops": peak64,
        "frac_fp64": flops64 / (ms_it64 * 1e-3) / 1e12 / peak64,
        "achieved_gbs": bytes64 / (ms_it64 * 1e-3) / 1e9,
        "frac_hbm": bytes64 / (ms_it64 * 1e-3) / 1e9 / load_peaks()[0],
        "ms_per_iteration": ms_it64, "flops_per_pixel_iteration": fp64_ops_inner(p.k, E),
        "bytes_per_pixel_iteration": bytes_inner_fp64(p.k, E),
        "kernels": ["k_inner_apply<%d,%d,%d,double>" % (p.k, p.m, E),
                    "k_inner_update<%d,%d,%d,double>" % (p.k, p.m, E)],
        "peak_source": "cuBLAS DGEMM 4096^3 through torch, best of 5 (CUDA events), measured "
                       "in this run; clocks as sampled for the line",
        "timing": "CUDA events around every launch in one profiled FP64 solve"}

    # ---- stand-alone operator apply (FP32), inputs larger than L2 ----------------------------
    X32 = X.to(torch.float32)
    for _ in range(3):
        Yap = op.apply(X32)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    barrier()
    a0.record(stream)
    for _ in range(reps):
        Yap = op.apply(X32)
    a1.record(stream)
    barrier()
    ms_apply = a0.elapsed_time(a1) / reps
    apply_bytes = bytes_apply(p.k, p.m, E) * p.n
    peak, peak_kind = load_peaks()
    apply_gbs = apply_bytes / (ms_apply * 1e-3) / 1e9

    # ---- roofline of the dominant kernel (from the timed steps' events) ---------------------
    # kernel time summed over every launch of the timed solves (including the few launches at
    # the end of a graph chunk that find nothing left to do), divided by the launches that
    # did work (one per inner iteration): a conservative per-launch time
    tot_apply = sum(i["ms_apply"] for i in infos)
    tot_update = sum(i["ms_update"] for i in infos)
    n_ap = n_up = sum(i["iterations"] for i in infos)
    shape = f"{p.k},{p.m},{E}" if E else f"{p.k},0,0"
    if tot_apply >= tot_update:
        kname = kernel_name("apply", last["apply_staged"], p.k, p.m, E)
        avg_ms, per_px = tot_apply / n_ap, bytes_inner_apply(p.k, p.m, E)
    else:
        kname = kernel_name("update", last["update_staged"], p.k, p.m, E)
        avg_ms, per_px = tot_update / n_up, bytes_inner_update(p.k, p.m)
    achieved = per_px * p.n / (avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "kernel": kname,
                # the recorded capture is of the row-major 1024 x 2048 workload only
                "traffic": (profiled_traffic(kname) if p.name == "sphere1024x2048_k6_m9"
                            else None),
                "bytes_per_launch": per_px * p.n, "avg_launch_ms": avg_ms,
                "launches_timed": n_ap, "launches_issued": sum(i["n_update"] for i in infos),
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                "timing": "CUDA events around every launch, in a pass of the same K solves "
                          "run right after the timed region"}

    # ---- end to end through the public API with host buffers --------------------------------
    # sylv_solve_host: the observations come from page-locked host memory and the solution goes
    # back to it inside the call (copies overlapped with the right-hand side and with the
    # refinement steps' residuals; the solution is copied after every update X += d)
    Xh = torch.empty((1, p.k, p.n), dtype=torch.float64).pin_memory()
    for _ in range(2):
        op.solve_host(Yh, out=Xh, tol=1e-8)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    g0.record(stream)
    d2h_copies = 0
    for _ in range(args.steps):
        _, info_h = op.solve_host(Yh, out=Xh, tol=1e-8)
        d2h_copies += max(int(info_h["outer"]), 1)
    g1.record(stream)
    barrier()
    ms_e2e = g0.elapsed_time(g1) / args.steps
    ms_e2e = max_over_ranks(ms_e2e, dist, dev)

    # ---- CPU oracle baseline (rank 0, N = 1) -------------------------------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_pcg_full(p)

    if rank == 0:
        line = {
            "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded sphere maps shaped like Planck: GMRF-smooth sources, "
                    "lognormal noise, power-law mixing)",
            "config": main_config(p),
            "precision": "mixed (FP32 inner PCG, FP64 refinement)",
            "iterations": last["iterations"], "outer": last["outer"],
            "relres": last["relres"],
            "autotune": {"tile": last["tile"], "slots_mult": last["slots_mult"],
                         "apply_staged": last["apply_staged"],
                         "update_staged": last["update_staged"],
                         "force_env": "SYLV_TUNE_FORCE=%d,%d,%d,%d" % (
                             last["tile"], last["slots_mult"], last["apply_staged"],
                             last["update_staged"])},
            "setup_ms": setup_ms,
            "rhs": {"ms": ms_rhs, "gbs": rhs_bytes / (ms_rhs * 1e-3) / 1e9},
            "fp64_pcg": {"ms": ms64, "iterations": info64["iterations"],
                         "relres": info64["relres"], "speedup_mixed": ms64 / ms,
                         "relerr_mixed_vs_fp64": relerr_mixed_vs_fp64,
                         "roofline": fp64_roof},
            "apply": {"ms": ms_apply, "gbs": apply_gbs, "frac": apply_gbs / peak,
                      "bytes": apply_bytes, "dtype": "f32"},
            "roofline": roofline,
            "kernel_ms_per_solve": {"inner_apply": tot_apply / len(infos),
                                    "inner_update": tot_update / len(infos),
                                    "residual64": sum(i["ms_residual"] for i in infos)
                                    / len(infos)},
            "e2e": {"value": ms_e2e, "unit": "ms",
                    "h2d_bytes_per_step": int(Yh.numel() * 8),
                    "d2h_bytes_per_step": int(Xh.numel() * 8 * d2h_copies / args.steps),
                    "api": "sylv_solve_host (Operator.solve_host)"},
            "gpu_launches": launches_timed,
            "ms_per_step_profiled": ms_profiled,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    op.close()


def make_operator(p, device=None):
    from paper_2204_08057_gb300.operator import Operator
    A = getattr(p, "A", None)
    return Operator(rowptr=p.graph.rowptr, col=p.graph.col, val=p.graph.val, D=p.D, tau=p.tau,
                    kappa=p.kappa, nu=None if A is not None else p.nu,
                    beta=None if A is not None else p.beta, A=A,
                    prior=getattr(p, "prior", "gmrf"))


def run_profile_case(args):
    """One solve (no graphs, polls every 4 iterations) and three FP32 applies of the workload:
    the launches an ncu capture of the inner kernels looks at."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    if args.separable:
        # one mixed block-Lanczos Sylvester solve of the separable workload (direct launches)
        p = synth.separable_problem(args.config, scale=args.scale if args.scale > 1 else None)
        op = make_operator(p)
        B = op.rhs(torch.from_numpy(p.Yobs).cuda())
        X, info = op.solve_sylvester(B, tol=p.tol, use_graph=0, check_every=4)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": p.name, "info": info}), flush=True)
        op.close()
        return
    p = with_order(synth.config_problem(args.config, scale=args.scale), args.pixel_order)
    op = make_operator(p)
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    X, info = op.solve(B, tol=p.tol, use_graph=0, check_every=4)
    X32 = X.to(torch.float32)
    for _ in range(3):
        op.apply(X32)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": p.name, "info": info}), flush=True)
    op.close()


def _timed(stream, fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def _base_line(args, metric, value, unit, config, higher=False):
    return {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value, "higher_is_better": higher,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded sphere maps shaped like Planck: GMRF-smooth sources, "
                    "power-law or printed mixing)", "config": config}


def run_batched(args):
    """64 independent lattice systems (sides 128..1024, k in 3..6, m = k + 2) in one
    sylv_solve_batched call vs the same systems solved one by one and vs FP64 batched.
    Under torchrun the 64 systems are split across the ranks (balanced on pixels x sources,
    no collective on the data path): each rank solves its subset in one batched call and the
    value is the slowest rank's time for the whole batch (total work fixed: strong scaling)."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    from paper_2204_08057_gb300.operator import solve_batched
    from paper_2204_08057_gb300.partition import partition_batch
    _build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    shapes = synth.batch_shapes(64)
    parts = partition_batch([s * s * k for s, k in shapes], world)
    mine = parts[rank]
    probs = synth.batch_problems(64, indices=mine)
    ops = [make_operator(p) for p in probs]
    Bs = [op.rhs(torch.from_numpy(p.Yobs).cuda()) for op, p in zip(ops, probs)]
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, precision=1)
    for _ in range(args.warmup):
        Xs, infos = solve_batched(ops, Bs, **kw)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    barrier()
    ms, (Xs, infos) = _timed(stream, lambda: solve_batched(ops, Bs, **kw), args.steps)
    barrier()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ms, dist, torch.device("cuda", local_rank))
    assert all(i["status"] == 0 for i in infos), infos
    # kernel times: one more call with CUDA events around every launch (outside the timed
    # region; profiling runs the shape groups one after another on one stream)
    _, infos_p = solve_batched(ops, Bs, profile=1, **kw)
    extra = {}
    if world == 1:
        for op, b in zip(ops, Bs):
            op.solve(b, tol=1e-8)
        ms_seq, _ = _timed(stream, lambda: [op.solve(b, tol=1e-8) for op, b in zip(ops, Bs)], 1)
        solve_batched(ops, Bs, tol=1e-8, precision=0)
        ms64, (X64, i64) = _timed(stream, lambda: solve_batched(ops, Bs, tol=1e-8, precision=0),
                                  1)
        rel = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
                  for a, b in zip(Xs, X64))
        extra = {"sequential_ms": ms_seq, "speedup_vs_sequential": ms_seq / ms,
                 "fp64_batched_ms": ms64, "speedup_vs_fp64": ms64 / ms,
                 "max_relerr_mixed_vs_fp64": rel}
    ntot = sum(s * s for s, _ in shapes)
    line = _base_line(args, "batched solve time to relres 1e-8 (64 systems, one call)", ms, "ms",
                      {"workload": "batch64_lattice128-1024_k3-6", "systems": len(shapes),
                       "total_pixels": ntot, "tol": 1e-8, "precision": "mixed"})
    line.update(extra)
    line.update({
        "n_gpus": world, "scaling": "strong" if world > 1 else "weak",
        "partition": {"systems_per_rank": [len(q) for q in parts],
                      "work_per_rank": [sum(shapes[i][0] ** 2 * shapes[i][1] for i in q)
                                        for q in parts],
                      "rule": "largest first to the least-loaded rank, work = n k"},
        "iterations_max": max(i["iterations"] for i in infos),
        "relres_max": max(i["relres"] for i in infos),
        "per_system": {"n": [p.n for p in probs], "k": [p.k for p in probs],
                       "iterations": [i["iterations"] for i in infos],
                       "outer": [i["outer"] for i in infos]},
        "kernel_ms_per_solve": {"inner_apply": infos_p[0]["ms_apply"],
                                "inner_update": infos_p[0]["ms_update"],
                                "residual64": infos_p[0]["ms_residual"],
                                "timing": "CUDA events around every launch, one extra call "
                                          "after the timed region"},
        "gpu_launches": infos[0]["launches"], "clocks": clk,
    })
    if rank == 0:
        print(json.dumps(line), flush=True)
    for op in ops:
        op.close()
    if dist is not None:
        dist.destroy_process_group()


def run_differentiable(args):
    """Forward solve plus adjoint solve and gradient reduction (loss ||X - X_true||^2) on the
    512 x 1024 sphere, k = 4, m = 7."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    p = synth.config_problem(4, scale=args.scale)
    op = make_operator(p)
    Y = torch.from_numpy(p.Yobs).cuda()
    Xt = torch.from_numpy(p.X_true).cuda()[None]
    stream = torch.cuda.current_stream()

    def step():
        X, info = op.solve(op.rhs(Y), tol=1e-8)
        gt, gk, gb, lam, info2 = op.backward(X, 2.0 * (X - Xt), Y, tol=1e-8)
        return X, gt, gk, gb, info, info2

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms, out = _timed(stream, step, args.steps)
    clk = clocks.stop() if clocks else None
    X, gt, gk, gb, info, info2 = out
    line = _base_line(args, "forward + adjoint gradient step time (tol 1e-8)", ms, "ms",
                      {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "tol": 1e-8})
    line.update({"forward_iterations": info["iterations"],
                 "adjoint_iterations": info2["iterations"],
                 "g_tau": list(map(float, gt)), "g_kappa": list(map(float, gk)),
                 "g_beta": list(map(float, gb)), "clocks": clk})
    print(json.dumps(line), flush=True)
    op.close()


def run_multirhs(args):
    """8 right-hand sides solved together on the 4096 x 12288 sphere (n = 50,331,648, k = 6,
    m = 9): the operator, noise maps and preconditioner are read once per tile for all of
    them.  Reports the solve time, the per-right-hand-side time and the stand-alone apply."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    p = synth.config_problem(5, scale=args.scale)
    gen_s = time.perf_counter() - t0
    op = make_operator(p)
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, precision=1)
    for _ in range(args.warmup):
        X, info = op.solve(B, **kw)
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms, (X, info) = _timed(stream, lambda: op.solve(B, **kw), args.steps)
    clk = clocks.stop() if clocks else None
    assert info["code"] == 0, info
    # kernel times: one more solve with CUDA events around every launch (outside the timed
    # region)
    del X
    X, info_p = op.solve(B, profile=1, **kw)
    X32 = X.to(torch.float32)
    del X
    for _ in range(2):
        op.apply(X32)
    ms_apply, _ = _timed(stream, lambda: op.apply(X32), 5)
    E = int(np.max(np.diff(p.graph.rowptr))) - 1
    apply_bytes = bytes_apply(p.k, p.m, E, R=p.nrhs) * p.n
    peak, _ = load_peaks()
    its = info["iterations"]
    # per pixel and iteration: the vectors of every right-hand side plus the operator data
    # (noise maps, ELL, diagonal, preconditioner factor) once, as the tile-major units read
    # it from HBM once and from L2 for the other right-hand sides
    op_apply = (p.m + E + 1) * 4 + 4 * E
    op_update = 4 * p.k + 2 * (p.k * (p.k + 1) // 2)
    per_px_it = (p.nrhs * (bytes_inner_apply(p.k, p.m, E) - op_apply) + op_apply
                 + p.nrhs * (bytes_inner_update(p.k, p.m) - op_update) + op_update)
    line = _base_line(args, "multi-RHS solve time to relres 1e-8 (8 right-hand sides together)",
                      ms, "ms", {"workload": p.name, "n": p.n, "k": p.k, "m": p.m,
                                 "nrhs": p.nrhs, "tol": 1e-8, "precision": "mixed"})
    line.update({
        "ms_per_rhs": ms / p.nrhs, "iterations": its, "outer": info["outer"],
        "relres_max": info["relres"],
        "kernel_ms_per_solve": {"inner_apply": info_p["ms_apply"],
                                "inner_update": info_p["ms_update"],
                                "residual64": info_p["ms_residual"],
                                "timing": "CUDA events around every launch, one extra solve "
                                          "after the timed region"},
        "inner_gbs": per_px_it * p.n * info_p["iterations"] /
                     ((info_p["ms_apply"] + info_p["ms_update"]) * 1e-3) / 1e9,
        "apply": {"ms": ms_apply, "gbs": apply_bytes / (ms_apply * 1e-3) / 1e9,
                  "frac": apply_bytes / (ms_apply * 1e-3) / 1e9 / peak, "nrhs": p.nrhs},
        "autotune": {"tile": info["tile"], "slots_mult": info["slots_mult"],
                     "apply_staged": info["apply_staged"], "update_staged": info["update_staged"]},
        "input_generation_s": gen_s, "clocks": clk, "gpu_launches": info["launches"],
    })
    print(json.dumps(line), flush=True)
    op.close()


def bytes_lanczos_a(k, E, s=4):
    """Pass A of a Lanczos step per pixel: raw block V_s (its neighbours come from cache) and
    V_{s-1}, write W, plus ELL values and columns, Laplacian diagonal, nu and 1/nu."""
    return (3 * k + E + 3) * s + 4 * E


def bytes_lanczos_b(k, s=4):
    """Pass B per pixel: read W and V_s, write V_{s+1}, plus nu."""
    return (3 * k + 1) * s


class DeviceMemory:
    """Device memory the library allocated between marks: the drop in cudaMemGetInfo's free
    bytes minus the growth of torch's reserved pool over the same interval."""

    def __init__(self):
        import torch
        torch.cuda.synchronize()
        self.last = self._now()
        self.marks = {}

    @staticmethod
    def _now():
        import torch
        free, _ = torch.cuda.mem_get_info()
        return free, torch.cuda.memory_reserved()

    def mark(self, name):
        import torch
        torch.cuda.synchronize()
        now = self._now()
        if name is not None:
            self.marks[name] = int((self.last[0] - now[0]) - (now[1] - self.last[1]))
        self.last = now

    def get(self, name):
        return self.marks.get(name)


def run_sylvester(args):
    """Separable special case of the workload (noise d_ci = t_c nu_i, one prior shape): time
    to relres 1e-8 of the block-Lanczos Sylvester solver (mixed and FP64) against the
    preconditioned CG (mixed and FP64) on the same system, and against CG with no
    preconditioner on the Kronecker-structured system, the comparison of Sec. 4 (one solve
    each; thousands of iterations)."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    p = synth.separable_problem(args.config, scale=args.scale if args.scale > 1 else None)
    mem = DeviceMemory()
    op = make_operator(p)
    mem.mark("handle")
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    stream = torch.cuda.current_stream()
    E = int(np.max(np.diff(p.graph.rowptr))) - 1
    # the FP32 Lanczos run reaches 1e-5 in one restart, which saves one FP64 residual and one
    # restart against the default 1e-4 (measured: 154 steps in 2 runs against 163 in 3)
    kw = dict(tol=1e-8, profile=0)

    def lz(prec, **extra):
        return op.solve_sylvester(B, precision=prec, inner_tol=1e-5, **{**kw, **extra})

    def cg(prec):
        return op.solve(B, precision=prec, **kw)

    mem.mark(None)
    cg(1)
    mem.mark("pcg_mixed_workspace")
    lz(1)
    mem.mark("lanczos_mixed_workspace")

    def cg_plain(prec):
        from paper_2204_08057_gb300 import binding as _B
        return op.solve(B, precision=prec, precond=_B.SYLV_PRECOND_NONE, maxit=100000, **kw)

    for _ in range(args.warmup):
        lz(1)
        cg(1)
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms_lz, (X_lz, info_lz) = _timed(stream, lambda: lz(1), args.steps)
    clk = clocks.stop() if clocks else None
    ms_cg, (X_cg, info_cg) = _timed(stream, lambda: cg(1), args.steps)
    lz(0)
    ms_lz64, (X_lz64, info_lz64) = _timed(stream, lambda: lz(0), args.fp64_steps)
    ms_cg64, (_, info_cg64) = _timed(stream, lambda: cg(0), args.fp64_steps)
    ms_cgp, (_, info_cgp) = _timed(stream, lambda: cg_plain(1), 1)
    ms_cgp64, (_, info_cgp64) = _timed(stream, lambda: cg_plain(0), 1)
    for inf in (info_lz, info_cg, info_lz64, info_cg64, info_cgp, info_cgp64):
        assert inf["code"] == 0, inf
    # kernel breakdown from one more solve with CUDA events around every launch
    _, info_prof = lz(1, profile=1)
    its = info_prof["iterations"]
    peak, _ = load_peaks()
    ba = bytes_lanczos_a(p.k, E) * p.n
    bb = bytes_lanczos_b(p.k) * p.n
    ms_a = info_prof["ms_apply"] / max(its, 1)
    ms_b = info_prof["ms_update"] / max(its, 1)
    rel = float(torch.linalg.norm(X_lz - X_cg) / torch.linalg.norm(X_cg))

    def summary(ms, inf):
        return {"ms": ms, "iterations": inf["iterations"], "outer": inf["outer"],
                "relres": inf["relres"]}

    # bounded memory: a fresh handle whose basis budget holds 48 blocks (runs restart there)
    os.environ["SYLV_LZ_BASIS_MB"] = str(int(np.ceil(48 * p.k * p.n * 4 / 2 ** 20)) + 1)
    op_b = make_operator(p)
    mem.mark(None)
    op_b.solve_sylvester(B, precision=1, inner_tol=1e-5, **kw)
    mem.mark("lanczos_mixed_workspace_bounded")
    ms_lzb, (_, info_lzb) = _timed(stream, lambda: op_b.solve_sylvester(
        B, precision=1, inner_tol=1e-5, **kw), args.steps)
    del os.environ["SYLV_LZ_BASIS_MB"]
    op_b.close()
    block_bytes = p.k * p.n * 4
    steps_per_run = -(-info_lz["iterations"] // max(info_lz["outer"], 1))
    memory = {
        "handle_bytes": mem.get("handle"),
        "pcg_mixed_workspace_bytes": mem.get("pcg_mixed_workspace"),
        "lanczos_mixed_workspace_bytes": mem.get("lanczos_mixed_workspace"),
        "lanczos_basis_block_bytes": block_bytes,
        "lanczos_steps_per_run": steps_per_run,
        "lanczos_basis_bytes_used": steps_per_run * block_bytes,
        "bounded": {"workspace_bytes": mem.get("lanczos_mixed_workspace_bounded"),
                    "basis_blocks": 48, "ms": ms_lzb, "iterations": info_lzb["iterations"],
                    "runs": info_lzb["outer"]},
        "how": "cudaMemGetInfo deltas around each first call, minus what torch's allocator "
               "reserved meanwhile; the basis is allocated to its capacity (up to 384 blocks "
               "or 60 % of free memory) at the first Lanczos call",
    }

    line = _base_line(args, "solve time to relres 1e-8, separable special case "
                            "(block-Lanczos Sylvester solver, mixed)", ms_lz, "ms",
                      {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "nrhs": 1,
                       "tol": 1e-8, "kappa0": float(p.kappa[0]), "lanczos_inner_tol": 1e-5,
                       "l2": "inputs larger than L2"})
    line.update({
        "lanczos_mixed": summary(ms_lz, info_lz),
        "lanczos_fp64": summary(ms_lz64, info_lz64),
        "pcg_mixed": summary(ms_cg, info_cg),
        "pcg_fp64": summary(ms_cg64, info_cg64),
        "cg_mixed_no_preconditioner": summary(ms_cgp, info_cgp),
        "cg_fp64_no_preconditioner": summary(ms_cgp64, info_cgp64),
        "lanczos_time_share_of_cg": {"mixed": ms_lz / ms_cgp, "fp64": ms_lz64 / ms_cgp64,
                                     "note": "Sec. 4 compares the Sylvester method with CG "
                                             "applied directly to the Kronecker system"},
        "memory": memory,
        "speedup_vs_pcg_mixed": ms_cg / ms_lz, "speedup_vs_pcg_fp64": ms_cg64 / ms_lz,
        "relerr_lanczos_vs_pcg": rel,
        "kernel_ms_per_solve": {"pass_a": info_prof["ms_apply"], "pass_b": info_prof["ms_update"],
                                "residual64_and_assembly": info_prof["ms_residual"],
                                "timing": "CUDA events around every launch, one extra solve"},
        "roofline": {"bound": "hbm",
                     "kernel": (f"k_lz_a_tma<{p.k},{E}>" if info_prof.get("apply_staged")
                                else f"k_lz_a<{p.k},{E},float>"),
                     "achieved": ba / (ms_a * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": ba / (ms_a * 1e-3) / 1e9 / peak, "traffic": None,
                     "bytes_per_launch": ba, "ms_per_launch": ms_a,
                     "pass_b_gbs": bb / (ms_b * 1e-3) / 1e9},
        "gpu_launches": info_lz["launches"], "clocks": clk,
    })
    print(json.dumps(line), flush=True)
    op.close()


def run_paper_model(args):
    """The paper's model (App. B mixing and weights, App. C intrinsic GMRF prior phi L^2) on the
    1024 x 2048 sphere: time to relres 1e-8 by mixed PCG, FP64 PCG and mixed Lanczos-Sylvester
    (the model is separable: C = T kron N, one prior shape), and by CG with no preconditioner
    on the Kronecker-structured system, the method Sec. 4 compares the Sylvester solver with."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    p = synth.igmrf_problem(args.config, scale=args.scale if args.scale > 1 else None)
    t0 = time.perf_counter()
    op = make_operator(p)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    B = op.rhs(torch.from_numpy(p.Yobs).cuda())
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, profile=0)

    def cg(prec, **extra):
        return op.solve(B, precision=prec, **{**kw, **extra})

    def lz(prec, **extra):
        return op.solve_sylvester(B, precision=prec, inner_tol=1e-5, **{**kw, **extra})

    for _ in range(args.warmup):
        cg(1)
        lz(1)
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms, (X, info) = _timed(stream, lambda: cg(1), args.steps)
    clk = clocks.stop() if clocks else None
    ms_lz, (X_lz, info_lz) = _timed(stream, lambda: lz(1), args.steps)
    cg(0)
    ms64, (X64, info64) = _timed(stream, lambda: cg(0), args.fp64_steps)
    from paper_2204_08057_gb300 import binding as _B
    plain = dict(precond=_B.SYLV_PRECOND_NONE, maxit=100000)
    ms_p, (_, info_p) = _timed(stream, lambda: cg(1, **plain), 1)
    ms_p64, (_, info_p64) = _timed(stream, lambda: cg(0, **plain), 1)
    for inf in (info, info_lz, info64, info_p, info_p64):
        assert inf["code"] == 0, inf
    _, info_prof = cg(1, profile=1)
    E = int(op_degree(p))

    def summary(t, inf):
        return {"ms": t, "iterations": inf["iterations"], "outer": inf["outer"],
                "relres": inf["relres"]}

    line = _base_line(args, "solve time to relres 1e-8, the paper's model (physical mixing, "
                            "intrinsic GMRF prior), mixed PCG", ms, "ms",
                      {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "nrhs": 1, "tol": 1e-8,
                       "prior": "phi L^2, phi = %g" % p.tau[0],
                       "mixing": "App. B printed table", "prior_ell_width": E,
                       "l2": "inputs larger than L2"})
    line.update({
        "setup_ms": setup_ms,
        "pcg_mixed": summary(ms, info), "pcg_fp64": summary(ms64, info64),
        "lanczos_mixed": summary(ms_lz, info_lz),
        "cg_mixed_no_preconditioner": summary(ms_p, info_p),
        "cg_fp64_no_preconditioner": summary(ms_p64, info_p64),
        "lanczos_time_share_of_cg": {"mixed": ms_lz / ms_p,
                                     "note": "Sec. 4 compares the Sylvester method with CG "
                                             "applied directly to the Kronecker system"},
        "speedup_mixed_vs_fp64": ms64 / ms,
        "relerr_mixed_vs_fp64": float(torch.linalg.norm(X - X64) / torch.linalg.norm(X64)),
        "relerr_lanczos_vs_fp64": float(torch.linalg.norm(X_lz - X64) / torch.linalg.norm(X64)),
        "kernel_ms_per_solve": {"inner_apply": info_prof["ms_apply"],
                                "inner_update": info_prof["ms_update"],
                                "residual64": info_prof["ms_residual"],
                                "staged": [info_prof["apply_staged"], info_prof["update_staged"]],
                                "timing": "CUDA events around every launch, one extra solve"},
        "gpu_launches": info["launches"], "clocks": clk,
    })
    print(json.dumps(line), flush=True)
    op.close()


def run_variance(args):
    """Posterior variances diag(G^{-1}) of the 1024 x 2048 workload from S Rademacher probes
    (sylv_variance: probe solves 16 at a time by the multi-right-hand-side mixed PCG)."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    p = synth.config_problem(args.config, scale=args.scale if args.scale > 1 else None)
    op = make_operator(p)
    S = int(args.variance)
    Z = torch.from_numpy(synth.rademacher_probes(S, p.k, p.n, seed=2204)).cuda()
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, precision=1)
    for _ in range(max(1, args.warmup // 2)):
        op.variance(Z, **kw)
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms, (var, info) = _timed(stream, lambda: op.variance(Z, **kw), max(1, args.steps // 2))
    clk = clocks.stop() if clocks else None
    assert info["code"] == 0, info
    v = var[:, :p.n]
    line = _base_line(args, "posterior variances diag(G^-1) from %d probes (probe solves to "
                            "relres 1e-8, 16 at a time)" % S, ms, "ms",
                      {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "probes": S,
                       "tol": 1e-8, "precision": "mixed", "l2": "inputs larger than L2"})
    line.update({"ms_per_probe": ms / S, "iterations_max": info["iterations"],
                 "outer_max": info["outer"],
                 "variance_range": [float(v.min()), float(v.max())],
                 "gpu_launches": info["launches"], "clocks": clk})
    print(json.dumps(line), flush=True)
    op.close()


def run_variance_probing(args):
    """Posterior variances diag(G^{-1}) of the 1024 x 2048 workload by probing
    (sylv_variance_probing: one 0/1 probe per colour and source, made on the device, solved 16
    at a time): colourings with P and P/2 colours per side; the pixel-wise change between the
    two estimates is the error estimate of the coarser one and bounds that of the finer one
    from above when the couplings decay with distance."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    _build.build()
    torch.cuda.set_device(0)
    p = synth.config_problem(args.config, scale=args.scale if args.scale > 1 else None)
    op = make_operator(p)
    P = int(args.variance_probing)
    stream = torch.cuda.current_stream()
    kw = dict(tol=1e-8, precision=1)
    col_f = synth.grid_colouring(p.graph, P)
    col_c = synth.grid_colouring(p.graph, max(P // 2, 1))
    op.variance_probing(col_c, max(P // 2, 1) ** 2, **kw)          # warm-up (plans, tuner)
    clocks = ClockSampler(0) if not args.no_clocks else None
    if clocks:
        clocks.start()
        time.sleep(0.5)
    ms, (var, info) = _timed(stream, lambda: op.variance_probing(col_f, P * P, **kw), 1)
    clk = clocks.stop() if clocks else None
    ms_c, (var_c, info_c) = _timed(stream, lambda: op.variance_probing(col_c, max(P // 2, 1) ** 2,
                                                                       **kw), 1)
    assert info["code"] == 0 and info_c["code"] == 0, (info, info_c)
    v, vc = var[:, :p.n], var_c[:, :p.n]
    rel = (v - vc).abs() / v.abs()
    nprobe = P * P * p.k
    line = _base_line(args, "posterior variances diag(G^-1) by probing with a distance colouring "
                            "(%d probes, solves to relres 1e-8, 16 at a time)" % nprobe, ms, "ms",
                      {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "colours": P * P,
                       "probes": nprobe, "tol": 1e-8, "precision": "mixed",
                       "l2": "inputs larger than L2"})
    line.update({"ms_per_probe": ms / nprobe, "iterations_max": info["iterations"],
                 "variance_range": [float(v.min()), float(v.max())],
                 "all_positive": bool((v > 0).all()),
                 "error_estimate": {"max_rel_change_vs_half": float(rel.max()),
                                    "median_rel_change_vs_half": float(rel.median()),
                                    "coarse_colours": max(P // 2, 1) ** 2,
                                    "coarse_ms": ms_c,
                                    "per_source_max": [float(x) for x in rel.max(dim=1).values]},
                 "gpu_launches": info["launches"], "clocks": clk})
    print(json.dumps(line), flush=True)
    op.close()


def run_learn(args):
    """Parameter learning on the 512 x 1024 sphere (k = 4, m = 7): N gradient steps over
    (log tau, log kappa, beta) on ||X - X_true||^2, each a parameter update in place, the
    right-hand side, a forward solve, an adjoint solve and the gradient reduction; with warm
    starts (the previous step's X and lambda) against cold starts."""
    import torch
    import synth
    from paper_2204_08057_gb300 import build as _build
    from paper_2204_08057_gb300.learn import HyperLearner
    _build.build()
    torch.cuda.set_device(0)
    p = synth.config_problem(4, scale=args.scale if args.scale > 1 else None)
    op = make_operator(p)
    Y = torch.from_numpy(p.Yobs).cuda()
    Xt = torch.from_numpy(p.X_true).cuda()[None]

    def loss_grad(X):
        d = X - Xt
        return float(torch.sum(d * d)), 2.0 * d

    stream = torch.cuda.current_stream()
    tau0, kappa0, beta0 = p.tau * 1.5, p.kappa * 0.7, p.beta + 0.05
    N = int(args.learn)
    out = {}
    for warm in (True, False):
        # steps of length 0.02 in (log tau, log kappa, beta) along the negative gradient
        kwl = dict(lr=0.02, normalize=True, warm=warm, tol=1e-8)
        hl = HyperLearner(op, Y, loss_grad, tau0, kappa0, beta0, **kwl)
        hl.step()                                  # warm-up (first step is cold either way)
        hl = HyperLearner(op, Y, loss_grad, tau0, kappa0, beta0, **kwl)
        ms, _ = _timed(stream, lambda: [hl.step() for _ in range(N)], 1)
        recs = hl.history
        out[warm] = {"ms_per_step": ms / N,
                     "forward_iterations": [r["forward_iterations"] for r in recs],
                     "adjoint_iterations": [r["adjoint_iterations"] for r in recs],
                     "loss": [r["loss"] for r in recs]}
    line = _base_line(args, "parameter-learning step (set params, rhs, forward + adjoint solve "
                            "to relres 1e-8, gradient), warm-started", out[True]["ms_per_step"],
                      "ms", {"workload": p.name, "n": p.n, "k": p.k, "m": p.m, "steps": N,
                             "tol": 1e-8, "precision": "mixed"})
    line.update({"warm": out[True], "cold": out[False],
                 "speedup_warm_vs_cold": out[False]["ms_per_step"] / out[True]["ms_per_step"]})
    print(json.dumps(line), flush=True)
    op.close()


def op_degree(p):
    """Off-diagonals per row of the prior shape the operator uses (L, or L^2 for the IGMRF)."""
    import numpy as _np
    deg = int(_np.max(_np.diff(p.graph.rowptr))) - 1
    return 3 * deg if getattr(p, "prior", "gmrf") == "igmrf" else deg


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
        return
    if args.impl == "ours" and args.learn > 0:
        run_learn(args)
        return
    if args.impl == "ours" and args.variance > 0:
        run_variance(args)
        return
    if args.impl == "ours" and args.variance_probing > 0:
        run_variance_probing(args)
        return
    if args.impl == "ours" and args.paper_model:
        run_paper_model(args)
        return
    if args.impl == "ours" and args.separable:
        run_sylvester(args)
        return
    if args.impl == "ours" and args.config in (3, 4, 5):
        {3: run_batched, 4: run_differentiable, 5: run_multirhs}[args.config](args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
