#!/usr/bin/env python3
"""Benchmark: Mpix/s per full IRLS unwrap of a 4096 x 4096 synthetic interferogram.

One step = one full unwrap (Alg. 1 with Alg. 2): 20 IRLS iterations, delta = 1e-3, tau = 1e-2,
CG tolerance 1e-6, coherence-derived weights, on the mixed-precision workload (ramp 0-800 rad,
80 bumps, 20 % low-coherence patches with noise 1.2 rad, two 3 pi steps).  Inputs stay resident
in HBM; the workspace (about 1.5 GB) is far larger than the 129 MB L2, so no flush is needed
between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank unwraps its own image (replicas: an unwrap does not shard) and the
value is the total pixel rate over ranks, timed by the slowest rank.  With `--workload batched`
the ranks split one set of 64 tiles per GPU by estimated cost (longest processing time first)
and each unwraps its share as one batch.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

OUTER, DELTA, TAU, CG_TOL = 20, 1e-3, 1e-2, 1e-6
# Total CG iterations of the 20-step unwrap of this workload as measured on the GPU (the oracle
# follows the same trajectory); used only to extrapolate the oracle's timed sample when no GPU
# run is available in the same process (the reference arm).
# CG iterations of the full unwrap the reference arm extrapolates to: 4096 x 4096 is the count
# measured for this workload (20 outer steps, cg_tol 1e-6: 4466 in split bf16, 4472 in float32);
# other sizes take a round figure
CG_TOTAL_REFERENCE = {4096: 4466, 2048: 3000}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def metric_name(n, w, schedule="fixed"):
    """The metric string of the single-image arms (the headline one at 4096 x 4096)."""
    size = f"{n}^2" if w == n else f"{n}x{w}"
    what = "matched L1 objective" if schedule == "fixed" else "CG schedule of Sec. 4.3"
    return f"Mpix/s per full IRLS unwrap at {size} ({what})"


def workload_name(n, prec, w=None):
    w = n if w is None else w
    m = max(n, w)
    return (f"irls_unwrap_{n}x{w}: synthetic interferogram (ramp 0-{800 * m // 4096} rad, "
            f"{max(1, round(80 * m / 4096))} bumps, 20% low-coherence patches, two 3pi steps), "
            f"coherence weights, {OUTER} IRLS iterations, delta {DELTA:g}, tau {TAU:g}, "
            f"cg_tol {CG_TOL:g}, DCT preconditioner {prec}")


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self):
        """Drops the samples taken so far: the sampler is started a second before the timed
        region (so that nvidia-smi's own start-up does not compete with the host thread that
        issues the kernels), and only samples from the timed region on are kept."""
        time.sleep(1.0)
        self.lines = []

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen (hw_slowdown,
    hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap) from `nvidia-smi --format=csv,
    noheader,nounits` lines of ClockSampler.Q.  Lines without all fields are skipped; a line
    whose clocks do not parse still reports its throttle reasons."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
        try:
            a, b = float(parts[1]), float(parts[2])
        except ValueError:
            continue
        sm.append(a)
        smax.append(b)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# CPU oracle sample (the cpu_baseline leg and the reference arm)
# ------------------------------------------------------------------------------------------
def oracle_sample(X, coh, cg_iters=2):
    """Times the FP64 oracle on the full-size image: problem set-up (gradients, weights, b, DCT
    bases), one outer step's reweighting + initial residual + first preconditioner application,
    then `cg_iters` PCG iterations.  Returns (t_setup, t_outer, t_iter) in seconds."""
    import oracle.irls as O
    t0 = time.perf_counter()
    pb = O.Problem(X, coh, tau=TAU)
    t1 = time.perf_counter()
    U = np.zeros((pb.N, pb.M))
    Vv, Vh = O.S_op(U) - pb.Gv, O.T_op(U) - pb.Gh
    Wv, Wh = O.reweight(Vv, Vh, pb.Cv, pb.Ch, DELTA)
    dv, dh = O.diag_d(pb.Cv, pb.Ch, Wv, Wh)
    t2 = time.perf_counter()
    O.pcg((U, Vv, Vh), pb.b, dv, dh, TAU, pb.basis_N, pb.basis_M, 0.0, 0)
    t3 = time.perf_counter()
    O.pcg((U, Vv, Vh), pb.b, dv, dh, TAU, pb.basis_N, pb.basis_M, 0.0, cg_iters)
    t4 = time.perf_counter()
    # pcg with cg_max = n does: residual, n x (A p, update) and n-1 preconditioner applications
    # plus the initial one; the per-iteration cost is the difference over n iterations
    t_iter = ((t4 - t3) - (t3 - t2)) / cg_iters
    return t1 - t0, (t2 - t1) + (t3 - t2), t_iter


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def extrapolated_oracle_rate(n, t_setup, t_outer, t_iter, cg_total, outer=OUTER, w=None):
    t_full = t_setup + outer * t_outer + cg_total * t_iter
    return (n * (n if w is None else w) / 1e6) / t_full, t_full


# ------------------------------------------------------------------------------------------
# Evaluation of results (measurement only; the solver's own statistics are float32 sums)
# ------------------------------------------------------------------------------------------
def l1_fp64(U, X, coh):
    """The L1 objective of problem (main), Sec. 2, of an unwrapped U, evaluated in FP64 on the
    host: wrapped float32 gradients of X, edge weights = mean of the two end-pixel coherences."""
    U = np.asarray(U, dtype=np.float64)
    X = np.asarray(X, dtype=np.float32)
    c = np.asarray(coh, dtype=np.float64)
    two_pi = np.float32(2.0 * np.pi)

    def wrap(d):
        return (d - two_pi * np.rint(d / two_pi).astype(np.float32)).astype(np.float64)

    gv = wrap((X[1:, :] - X[:-1, :]).astype(np.float32))
    gh = wrap((X[:, 1:] - X[:, :-1]).astype(np.float32))
    cv = 0.5 * (c[1:, :] + c[:-1, :])
    ch = 0.5 * (c[:, 1:] + c[:, :-1])
    return float(np.sum(cv * np.abs(U[1:, :] - U[:-1, :] - gv)) +
                 np.sum(ch * np.abs(U[:, 1:] - U[:, :-1] - gh)))


def k_agreement(U1, U2):
    """Share of pixels whose 2pi multiple of U1 - U2 (less its circular mean) is the most common
    one: 1.0 when two unwraps of the same image differ by a constant only."""
    d = np.asarray(U1, dtype=np.float64) - np.asarray(U2, dtype=np.float64)
    c = float(np.angle(np.sum(np.exp(1j * d))))
    k = np.rint((d - c) / (2.0 * np.pi)).astype(np.int64)
    _, cnt = np.unique(k, return_counts=True)
    return float(cnt.max() / k.size)


def measure_forms(d, X, C, timed_unwraps=2):
    """The other forms of the same 4096 x 4096 unwrap (and the 64-tile batch), each timed with
    CUDA events after one warm-up unwrap (the plain float32 form: one unwrap, no warm-up), with
    the final L1 objective evaluated in FP64 on each result.  Not part of `value`."""
    import torch
    import paper_2401_09961_gb300 as irls
    import synthetic
    stream = torch.cuda.current_stream()
    H, W = X.shape
    out = {}

    def timed(run, n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n):
            r = run()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / n, r

    single = [("fp32_plain_simt_dct", dict(precision="fp32"), 0, 1),
              ("fp32_fft_dct", dict(precision="fp32", dct_form="fft"), 1, timed_unwraps),
              ("fp32_fft_dct_u_only_system", dict(precision="fp32", dct_form="fft",
                                                  system="schur"), 1, timed_unwraps),
              ("fp16_folded", dict(precision="fp16"), 1, timed_unwraps),
              ("bf16x3_folded_u_only_system", dict(precision="bf16x3", system="schur"), 1,
               timed_unwraps)]
    for name, kw, warm, n in single:
        with irls.Plan(H, W, tau=TAU, delta=DELTA, outer_iters=OUTER, cg_tol=CG_TOL,
                       cg_max_iter=1000, **kw) as p:
            U = torch.empty_like(X)
            for _ in range(warm):
                p.unwrap(X, C, out=U)
            t, (_, st) = timed(lambda: p.unwrap(X, C, out=U), n)
            out[name] = {"s_per_unwrap": t, "mpix_s": H * W / 1e6 / t, "unwraps_timed": n,
                         "cg_iters_total": st["cg_total"],
                         "l1_fp64": l1_fp64(U.cpu().numpy(), d["X"], d["coherence"])}
    shapes = synthetic.batched_tile_shapes(n=64, seed_base=1000)
    tiles = synthetic.batched_tiles(n=64, seed_base=1000, indices=list(range(64)))
    Xs = [torch.as_tensor(t["X"]).cuda() for t in tiles]
    Cs = [torch.as_tensor(t["coherence"]).cuda() for t in tiles]
    mpix = sum(h * w for h, w in shapes) / 1e6
    with irls.Batch(shapes, precision="bf16x3", tau=TAU, delta=DELTA, outer_iters=OUTER,
                    cg_tol=CG_TOL, cg_max_iter=1000) as b:
        b.autotune()
        b.unwrap(Xs, Cs)
        t, (_, st) = timed(lambda: b.unwrap(Xs, Cs), timed_unwraps)
        out["bf16x3_batched_64_tiles"] = {
            "s_per_batch": t, "mpix_s": mpix / t, "batches_timed": timed_unwraps,
            "mpix_per_batch": mpix, "cg_iters_total": sum(x["cg_total"] for x in st)}
    out["_note"] = ("same image and options as the headline (one warm-up, then CUDA-event "
                    "timing), single-image forms at the default stencil tiles (the headline's "
                    "and the batch's are autotuned); the batch is the 64-tile uneven-size "
                    "workload; l1_fp64 is the objective of "
                    "problem (main) evaluated in FP64 on each result")
    return out


# ------------------------------------------------------------------------------------------
def rank_max(x, world, device="cuda"):
    """x maximised over the ranks of the process group (the slowest rank's time); x at N = 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_sum(x, world, device="cuda"):
    """x summed over the ranks (the units every rank processed); x at N = 1."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--width", type=int, default=None,
                    help="image width (default: --size, a square image); e.g. --size 4000 "
                         "--width 16000 for the paper's 4000 x M scaling shapes")
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16", "bf16x3", "fp16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default stencil tile shapes (no timing pass before warm-up)")
    ap.add_argument("--dct-form", default="auto", choices=["auto", "direct", "folded", "fft"],
                    help="preconditioner form (auto: folded where allowed; fft: fast transforms "
                         "in float32, with --precision fp32)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "tiled", "adjoint"],
                    help="single: one 4096 x 4096 image per step (the benchmark); batched: 64 "
                         "tiles with sides in {256, ..., 1536} per step, one batched solve; "
                         "tiled: one --size x --width image cut into overlapping tiles solved "
                         "as one batch and stitched; adjoint: the 1024 x 1024 15-step forward "
                         "with its checkpoints and the adjoint sweep (dL/dX, dL/dcoherence)")
    ap.add_argument("--tile", type=int, default=1024, help="tile side of --workload tiled")
    ap.add_argument("--overlap", type=int, default=64, help="tile overlap of --workload tiled")
    ap.add_argument("--outer", type=int, default=OUTER,
                    help="IRLS iterations per unwrap (short profiling runs only; the benchmark "
                         "workload is 20); with --cg-schedule paper, the most it may take")
    ap.add_argument("--system", default="full", choices=["full", "schur"],
                    help="full: the paper's (U, V) system (the benchmark); schur: the U-only "
                         "system left after eliminating V")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the comparison of the other forms (plain float32, float16, U-only "
                         "system, 64-tile batch) after the headline at 4096 x 4096")
    ap.add_argument("--cg-schedule", default="fixed", choices=["fixed", "paper"],
                    help="fixed: every solve capped at 1000 CG iterations (the benchmark); paper: "
                         "the adaptive CG budget and IRLS stop of Sec. 4.3")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n = args.size
    prec = args.precision

    if args.impl == "reference":
        return reference_arm(args, rank, world, n, prec)
    if args.workload == "batched":
        return batched_arm(args, rank, world, local)
    if args.workload == "tiled":
        return tiled_arm(args, rank, world, local)
    if args.workload == "adjoint":
        return adjoint_arm(args, rank, world, local)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")

    import paper_2401_09961_gb300 as irls
    import synthetic
    import ctypes

    wd = args.width or n
    d = synthetic.config_4096_mixed(seed=20 + rank, H=n, W=wd)
    X = torch.as_tensor(d["X"]).cuda()
    C = torch.as_tensor(d["coherence"]).cuda()
    flexible = 1 if prec == "bf16" else 0
    plan = irls.Plan(n, wd, tau=TAU, delta=DELTA, outer_iters=args.outer, cg_tol=CG_TOL,
                     cg_max_iter=1000, precision=prec, flexible_cg=flexible,
                     cg_schedule=args.cg_schedule, system=args.system, dct_form=args.dct_form)
    stream = torch.cuda.current_stream()
    # stencil tile shapes timed on this GPU before the warm-up (outside the timed region)
    tune = None if (args.no_autotune or args.system != "full") else plan.autotune()
    U = torch.empty_like(X)
    for _ in range(args.warmup):
        _, st = plan.unwrap(X, C, out=U)
    torch.cuda.synchronize()

    # ---- timed region: K full unwraps, device-timed with events on the launching stream ----
    # (the live per-class profiler stays off here; its split comes from a separate pass below)
    L = irls.lib()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        _, st = plan.unwrap(X, C, out=U)
        stats.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # ---- per-class split: a separate pass with the live profiler on (not part of `value`) ----
    prof_steps = min(args.steps, 3)
    L.irls_plan_set_profiling(plan.handle, 1)
    for _ in range(prof_steps):
        plan.unwrap(X, C, out=U)
    torch.cuda.synchronize()
    prof_ms = (ctypes.c_double * 6)()
    prof_n = (ctypes.c_longlong * 6)()
    L.irls_plan_profile(plan.handle, prof_ms, prof_n, 6)
    L.irls_plan_set_profiling(plan.handle, 0)
    ms = rank_max(ms, world)
    ms_step = ms / args.steps
    mpix_step = n * wd / 1e6
    # every rank unwraps its own n x wd image: the whole job's pixels over the slowest rank's time
    value = rank_sum(mpix_step, world) * args.steps / (ms / 1e3)

    # ---- roofline of the dominant kernel class ----
    peaks, peak_src = load_peaks()
    P = n * wd
    cg_total = stats[-1]["cg_total"]
    outer_done = stats[-1]["outer_done"]
    classes = ["init", "reweight_residual", "direction_pap", "update", "dct_precond", "finalize"]
    per_cls = {c: {"ms": prof_ms[i], "launches": int(prof_n[i])} for i, c in enumerate(classes)}
    # live launches (skipped launches after CG stopped are excluded from the averages)
    live = {"direction_pap": cg_total * prof_steps, "update": cg_total * prof_steps,
            "dct_precond": (cg_total + outer_done) * prof_steps,
            "reweight_residual": outer_done * prof_steps, "finalize": outer_done * prof_steps}
    folded = plan.folded
    fft = plan.dct_form_name == "fft"
    # bf16 copy of r_U written for the direct tensor-core forms (hi, plus lo in split precision)
    emit = 0.0 if (prec == "fp32" or folded) else (4.0 if prec == "bf16x3" else 2.0)
    if args.system == "schur":
        # U-only kernels: direction reads z, p_old, D (2), writes p; update reads p, D (2), U,
        # r and writes U, r; reweighting reads U, V (2), C (2), G (2) and writes W (2), D (2), r
        bytes_px = {"direction_pap": 20.0, "reweight_residual": 48.0 + emit,
                    "update": 28.0 + emit + (4.0 if flexible else 0)}
    else:
        bytes_px = {"direction_pap": 44.0, "reweight_residual": 56.0 + emit,
                    "update": 68.0 + emit + (4.0 if flexible else 0)}
    # finalize: U, G (2), C (2), V (2), W (2) read; then U read and written by the mean removal
    bytes_px["finalize"] = 44.0
    # fast-transform preconditioner: three passes, each reading and writing one float32 plane
    if fft:
        bytes_px["dct_precond"] = 24.0
    for c in ("direction_pap", "update", "reweight_residual", "finalize") + (
            ("dct_precond",) if fft else ()):
        if per_cls[c]["ms"] > 0 and live.get(c):
            t = per_cls[c]["ms"] / 1e3 / live[c]
            per_cls[c].update({"ms_per_live_launch": t * 1e3, "bytes_per_px": bytes_px[c],
                               "achieved_gbs": bytes_px[c] * P / t / 1e9,
                               "frac_of_hbm": bytes_px[c] * P / t / 1e9 / peaks["hbm_gbs"]})
    per_cls["_pass"] = f"{prof_steps} unwraps with the live per-class profiler on, after the timed region"
    # multiply-adds the preconditioner performs per application: four n^3 products in the direct
    # form; the folded form runs each stage as half-size products (half of that)
    dct_flops = 4.0 * n * wd * (n + wd) * (0.5 if folded else 1.0)
    dom = max(("direction_pap", "update", "dct_precond", "reweight_residual"),
              key=lambda c: per_cls[c]["ms"])
    avg_s = per_cls[dom]["ms"] / 1e3 / max(live[dom], 1)
    if dom == "dct_precond" and not fft:
        if prec == "fp32":
            clk_mhz = clk.get("sm_mhz") or 1900.0
            peak = 152 * 128 * 2 * clk_mhz * 1e6 / 1e12
            roof = {"kernel": "dct_precond (4 SIMT fp32 GEMMs)", "bound": "alu",
                    "achieved": dct_flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "peak_source": f"152 SMs x 128 fp32 lanes x 2 x {clk_mhz:.0f} MHz (derived)"}
        else:
            sus = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            passes = 3 if prec == "bf16x3" else 1
            alg = dct_flops / avg_s / 1e12
            form = ("k_fold_r + k2_fold_fused: the four folded even/odd stages in one persistent "
                    "CTA-pair launch" if folded else "four grouped tcgen05 GEMMs, direct form")
            roof = {"kernel": f"dct_precond ({form}, {prec})", "bound": "tensor",
                    "achieved": alg, "peak": sus / passes, "unit": "TFLOP/s",
                    "peak_source": (f"bf16_tflops_sustained ({peak_src}) / {passes}: the split "
                                    "product issues three bf16 MMAs per multiply-add"
                                    if passes == 3 else
                                    f"bf16_tflops_sustained ({peak_src}); float16 and bf16 "
                                    "have the same dense tensor rate" if prec == "fp16" else
                                    f"bf16_tflops_sustained ({peak_src})"),
                    "tensor_pipe_frac_of_bf16_peak": alg * passes / sus}
    else:
        achieved = bytes_px[dom] * P / avg_s / 1e9
        name = ("dct_precond (k_fftdct_rows_fwd + k_fftdct_cols + k_fftdct_rows_inv: fast "
                "transforms, float32)" if dom == "dct_precond" else dom)
        roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "peak_source": f"hbm_gbs ({peak_src})"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["sm_mhz_median_timed_region"] = clk.get("sm_mhz")
    # DRAM bytes per preconditioner application (dram__bytes_read.sum + dram__bytes_write.sum
    # of k_fold_r, 85.5 MB, and k2_fold_fused, 779.2 MB) from one ncu capture of the current
    # kernels at 4096 x 4096, split bf16, folded form (the algorithmic traffic is 0.81 GB)
    measured_traffic = {(4096, 4096, "bf16x3", True): 864.7e6}
    roof["traffic"] = (measured_traffic.get((n, wd, prec, bool(folded)))
                       if dom == "dct_precond" else None)
    if roof["traffic"] is not None:
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, one "
                                  "application, k_fold_r + k2_fold_fused")
        # clock-independent tensor-pipe activity of k2_fold_fused from the same capture
        roof["ncu_tensor_pipe_active_pct"] = {"avg": 80.3, "max": 83.4, "min": 77.4,
                                              "sm_clock_ghz_under_ncu": 1.84}
    roof["avg_launch_ms"] = avg_s * 1e3
    kernels_per_class = {"init": 2, "reweight_residual": 1, "direction_pap": 1, "update": 1,
                         "dct_precond": 2 if folded else (3 if fft else 4), "finalize": 2}
    # launches of the timed region: the profiled pass ran the same kernels per unwrap
    gpu_launches = sum(per_cls[c]["launches"] * kernels_per_class[c] for c in classes)
    gpu_launches = gpu_launches * args.steps // max(prof_steps, 1) + args.steps  # + copy-out

    # ---- end to end through the public API with host (pinned) buffers ----
    e2e = None
    if not args.no_e2e:
        Xh = torch.as_tensor(d["X"]).pin_memory()
        Ch = torch.as_tensor(d["coherence"]).pin_memory()
        irls.unwrap(Xh, Ch, plan=plan)   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            Uh = irls.unwrap(Xh, Ch, plan=plan)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = rank_max(t_e2e, world)
        e2e = {"value": rank_sum(mpix_step, world) * args.steps / t_e2e, "unit": "Mpix/s",
               "h2d_bytes_per_step": int(Xh.numel() * 4 + Ch.numel() * 4),
               "d2h_bytes_per_step": int(Uh.numel() * 4)}

    # ---- CPU oracle baseline (rank 0, N = 1 only) ----
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        ts, to, ti = oracle_sample(d["X"], d["coherence"])
        rate, tfull = extrapolated_oracle_rate(n, ts, to, ti, cg_total, outer_done, wd)
        cpu = {"value": rate, "unit": "Mpix/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": (f"FP64 NumPy oracle on the full {n}x{wd} image: set-up + one outer step "
                          f"+ 2 PCG iterations timed ({ts:.1f} s, {to:.1f} s, {ti:.2f} s/iter), "
                          f"extrapolated to a full unwrap with this run's {cg_total} CG "
                          f"iterations: {tfull:.0f} s"),
               "extrapolated": True}

    # ---- the headline result's objective in FP64, and the other forms (rank 0, N = 1) ----
    l1_head = None
    forms = None
    if rank == 0 and world == 1:
        l1_head = l1_fp64(U.cpu().numpy(), d["X"], d["coherence"])
        if (not args.no_forms and n == 4096 and wd == 4096 and prec == "bf16x3"
                and args.system == "full" and args.cg_schedule == "fixed" and args.outer == OUTER):
            forms = measure_forms(d, X, C)
            forms["bf16x3_folded_headline"] = {"s_per_unwrap": ms_step / 1e3, "mpix_s": value,
                                               "cg_iters_total": cg_total, "l1_fp64": l1_head}

    if rank == 0:
        out = {
            "metric": metric_name(n, wd, args.cg_schedule),
            "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "fp32" else
            f"f32+{prec}-tensor-core-dct", "data": "synthetic",
            "config": {"workload": workload_name(n, "fp32 fast transforms" if fft else prec, wd),
                       "size": [n, wd],
                       "outer_iters": args.outer, "outer_done": outer_done,
                       "cg_schedule": args.cg_schedule, "system": args.system,
                       "delta": DELTA, "tau": TAU,
                       "cg_tol": CG_TOL,
                       "precision": prec, "flexible_cg": bool(flexible),
                       "dct_form": plan.dct_form_name,
                       "stencil_tiles": {"direction_rows": plan.tiles[0],
                                         "update_rows": plan.tiles[1],
                                         "autotuned": tune is not None},
                       "cg_iters_total": cg_total, "l1_objective": stats[-1]["l1_obj"][-1],
                       "l1_objective_fp64": l1_head,
                       "cg_iters_per_outer": stats[-1]["cg_iters"],
                       **({"cg_caps": stats[-1]["cg_cap"]} if args.cg_schedule == "paper"
                          else {}),
                       "parallelism": f"replicas x{world}",
                       "l2": "workspace > L2 (no flush needed)"},
            "roofline": roof,
            "kernel_classes": per_cls,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": gpu_launches,
            "clocks": clk,
            "forms": forms,
        }
        print(json.dumps(out))
    plan.close()
    if world > 1:
        dist.destroy_process_group()


def batched_arm(args, rank, world, local):
    """64 uneven tiles per GPU (sides from {256, ..., 1536}, tile t seeded 1000 + t) unwrapped
    together: one step = one batched solve of the rank's tiles, 20 outer steps each,
    split-bf16 preconditioner.  On N GPUs the job is the 64 N tiles 1000 ... 1000 + 64 N - 1,
    split across the ranks by longest-processing-time-first on the estimated cost of a tile,
    with no collective on the data path."""
    import torch
    import torch.distributed as dist
    import paper_2401_09961_gb300 as irls
    from paper_2401_09961_gb300 import sharding
    import synthetic
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    all_shapes = synthetic.batched_tile_shapes(n=64 * world, seed_base=1000)
    mine = sharding.shard_tiles(all_shapes, rank, world)
    tiles = synthetic.batched_tiles(n=64 * world, seed_base=1000, indices=mine)
    shapes = [d["X"].shape for d in tiles]
    Xs = [torch.as_tensor(d["X"]).cuda() for d in tiles]
    Cs = [torch.as_tensor(d["coherence"]).cuda() for d in tiles]
    mpix = sum(h * w for h, w in shapes) / 1e6
    prec = args.precision if args.precision != "fp32" else "bf16x3"
    if prec == "fp16":
        raise SystemExit("bench.py: the batched form runs bf16x3 or bf16 (float16 is single-image)")
    b = irls.Batch(shapes, precision=prec, tau=TAU, delta=DELTA, outer_iters=args.outer,
                   cg_tol=CG_TOL, cg_max_iter=1000, flexible_cg=1 if prec == "bf16" else 0,
                   dct_form=args.dct_form)
    # stencil tile shapes timed on this GPU before the warm-up (outside the timed region)
    tune = None if args.no_autotune else b.autotune()
    for _ in range(args.warmup):
        b.unwrap(Xs, Cs)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, st = b.unwrap(Xs, Cs)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    # each rank solves its own share of the tiles (its own pixel count)
    ms = rank_max(e0.elapsed_time(e1), world) / args.steps
    mpix_all = rank_sum(mpix, world)
    # the same tiles one at a time through single-image plans, for comparison
    t_single = 0.0
    if not args.no_e2e:
        for X, C, (h, w) in zip(Xs, Cs, shapes):
            with irls.Plan(h, w, precision=prec, tau=TAU, delta=DELTA, outer_iters=args.outer,
                           cg_tol=CG_TOL, cg_max_iter=1000,
                           flexible_cg=1 if prec == "bf16" else 0, dct_form=args.dct_form) as p:
                p.unwrap(X, C)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                p.unwrap(X, C)
                torch.cuda.synchronize()
                t_single += time.perf_counter() - t0
    if rank == 0:
        out = {
            "metric": "Mpix/s per batched IRLS unwrap of 64 uneven tiles",
            "value": mpix_all / (ms / 1e3), "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"f32+{prec}-tensor-core-dct", "data": "synthetic",
            "config": {"workload": f"{64 * world} tiles, sides in {{256,...,1536}} (non-square), "
                                   f"{mpix_all:.1f} Mpix total, {args.outer} IRLS iterations, "
                                   f"delta {DELTA:g}, tau {TAU:g}, cg_tol {CG_TOL:g}, {prec}",
                       "cg_iters_total": sum(x["cg_total"] for x in st),
                       "cg_iters_max_tile": max(x["cg_total"] for x in st),
                       "dct_form": "folded" if b.folded else "direct",
                       "stencil_tiles": {"direction_rows": b.tiles[0], "update_rows": b.tiles[1],
                                         "autotuned": tune is not None},
                       "uses_graphs": b.uses_graphs,
                       "sharding": ("none" if world == 1 else
                                    f"LPT over {world} ranks, rank 0 holds {len(mine)} tiles")},
            "single_image_sequential_mpix_s": (mpix / t_single) if t_single else None,
            "clocks": clk,
        }
        print(json.dumps(out))
    b.close()
    if world > 1:
        dist.destroy_process_group()


def tiled_arm(args, rank, world, local):
    """One --size x --width image of the mixed-coherence law per rank, cut into overlapping tiles
    (--tile, --overlap) solved as one batch and stitched (irls_unwrap_tiled); the same image
    through one single-image plan once, outside the timed region, for the integer-map agreement
    and the L1 objectives."""
    import torch
    import torch.distributed as dist
    import paper_2401_09961_gb300 as irls
    import synthetic
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    H, W = args.size, args.width or args.size
    d = synthetic.config_4096_mixed(seed=20 + rank, H=H, W=W)
    X = torch.as_tensor(d["X"]).cuda()
    C = torch.as_tensor(d["coherence"]).cuda()
    prec = args.precision if args.precision in ("bf16x3", "bf16") else "bf16x3"
    kw = dict(tau=TAU, delta=DELTA, outer_iters=args.outer, cg_tol=CG_TOL, cg_max_iter=1000,
              precision=prec, flexible_cg=1 if prec == "bf16" else 0, dct_form=args.dct_form)
    t = irls.Tiled(H, W, tile=args.tile, overlap=args.overlap, **kw)
    if not args.no_autotune:
        t.autotune()
    U = torch.empty_like(X)
    for _ in range(args.warmup):
        t.unwrap(X, C, out=U)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.mark()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, st, _ = t.unwrap(X, C, out=U)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = rank_max(e0.elapsed_time(e1), world) / args.steps
    mpix = rank_sum(H * W / 1e6, world)
    n_tiles, (th, tw) = t.n_tiles, t.tile_shape
    t.close()
    extra = {}
    if not args.no_e2e and rank == 0:
        with irls.Plan(H, W, **kw) as p:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Us, ss = p.unwrap(X, C)
            torch.cuda.synchronize()
            t_single = time.perf_counter() - t0
        Ut = U.cpu().numpy()
        Usn = Us.cpu().numpy()
        extra = {"single_plan_s": t_single, "single_plan_mpix_s": H * W / 1e6 / t_single,
                 "k_map_agreement_vs_single_plan": k_agreement(Ut, Usn),
                 "l1_tiled": l1_fp64(Ut, d["X"], d["coherence"]),
                 "l1_single_plan": l1_fp64(Usn, d["X"], d["coherence"])}
    if rank == 0:
        out = {
            "metric": f"Mpix/s per tiled IRLS unwrap of one {H}x{W} image",
            "value": mpix / (ms / 1e3), "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"f32+{prec}-tensor-core-dct",
            "data": "synthetic",
            "config": {"workload": workload_name(H, prec, W) + f", {n_tiles} tiles of "
                                   f"{th}x{tw} (overlap {args.overlap}) as one batch",
                       "cg_iters_total_all_tiles": sum(x["cg_total"] for x in st),
                       "cg_iters_max_tile": max(x["cg_total"] for x in st)},
            **extra,
            "clocks": clk,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def adjoint_arm(args, rank, world, local):
    """The differentiation workload: a 1024 x 1024 image of the adjoint law (ramp 0-200 rad, 20
    bumps, coherence weights), 15 IRLS steps recorded with their checkpoints, then the adjoint
    sweep for L = sum (U - mean U - U_ref)^2, U_ref the noise-free phase.  One step = forward
    with checkpoints + adjoint sweep, timed with CUDA events; the split-bf16 folded form, with
    the float32 dense and fast-transform forms measured after it (not part of `value`)."""
    import torch
    from paper_2401_09961_gb300.autograd import unwrap_backward, unwrap_record
    import paper_2401_09961_gb300 as irls
    import synthetic
    torch.cuda.set_device(local)
    n = 1024
    d = synthetic.config_adjoint_1024(seed=30 + rank)
    X = torch.as_tensor(d["X"]).cuda()
    C = torch.as_tensor(d["coherence"]).cuda()
    Uref = torch.as_tensor((d["phi_true"] - d["phi_true"].mean()).astype(np.float32)).cuda()
    stream = torch.cuda.current_stream()

    def run(plan):
        U, tape, st = unwrap_record(plan, X, C)
        dLdU = 2.0 * (U - U.mean() - Uref)
        e_mid = torch.cuda.Event(enable_timing=True)
        e_mid.record(stream)
        dX, dc, sb = unwrap_backward(tape, dLdU)
        tape.free()
        return e_mid, st, sb, dX

    def measure(kw, steps, warmup):
        with irls.Plan(n, n, tau=TAU, delta=DELTA, outer_iters=15, cg_tol=CG_TOL,
                       cg_max_iter=1000, **kw) as p:
            for _ in range(warmup):
                run(p)
            torch.cuda.synchronize()
            fwd = bwd = 0.0
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                e_mid, st, sb, dX = run(p)
                e1.record(stream)
                torch.cuda.synchronize()
                fwd += e0.elapsed_time(e_mid)
                bwd += e_mid.elapsed_time(e1)
            return {"form": p.dct_form_name, "forward_s": fwd / steps / 1e3,
                    "adjoint_s": bwd / steps / 1e3,
                    "mpix_s": n * n / 1e6 / ((fwd + bwd) / steps / 1e3),
                    "cg_forward": st["cg_total"], "cg_adjoint": sb["cg_total"],
                    "dldx_sum": float(dX.sum().item())}

    clocks = ClockSampler(local)
    clocks.start()
    clocks.mark()
    head = measure(dict(precision="bf16x3"), args.steps, args.warmup)
    clk = clocks.stop()
    others = {}
    if not args.no_forms:
        others["fp32_dense"] = measure(dict(precision="fp32"), 1, 0)
        others["fp32_fft"] = measure(dict(precision="fp32", dct_form="fft"), args.steps, 1)
    if rank == 0:
        out = {
            "metric": "Mpix/s per forward (15 IRLS steps, checkpointed) + adjoint sweep at 1024^2",
            "value": head["mpix_s"], "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * (head["forward_s"] + head["adjoint_s"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16x3-tensor-core-dct", "data": "synthetic",
            "config": {"workload": "1024x1024 adjoint law (ramp 0-200 rad, 20 bumps, noise 0.5 "
                                   "rad, coherence weights), 15 IRLS steps, delta 1e-3, tau 1e-2, "
                                   f"cg_tol {CG_TOL:g}; L = sum (U - mean U - U_ref)^2",
                       **head},
            "forms": others or None,
            "clocks": clk,
        }
        print(json.dumps(out))


def reference_arm(args, rank, world, n, prec):
    """The oracle as it stands on the host cores: each step times the bounded full-size sample
    of oracle_sample() and extrapolates it to one full unwrap."""
    if rank != 0:
        return
    import synthetic
    d = synthetic.config_4096_mixed(seed=20, H=n, W=n)
    cg_total = CG_TOTAL_REFERENCE.get(n, 5000)
    rates, fulls = [], []
    for s in range(args.warmup + args.steps):
        ts, to, ti = oracle_sample(d["X"], d["coherence"])
        r, tf = extrapolated_oracle_rate(n, ts, to, ti, cg_total)
        if s >= args.warmup:
            rates.append(r)
            fulls.append(tf)
    value = statistics.median(rates)
    sample = (f"FP64 NumPy oracle on the full {n}x{n} image: set-up + one outer step + 2 PCG "
              f"iterations per step, extrapolated to a full unwrap with {cg_total} CG iterations "
              f"(median {statistics.median(fulls):.0f} s per unwrap)")
    out = {
        "impl": "reference",
        "metric": metric_name(n, n),
        "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * (n * n / 1e6) / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(n, "fp64 dense (oracle)"), "size": [n, n]},
        "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": cpu_threads(),
                         "kind": "oracle", "sample": sample, "extrapolated": True},
        "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


if __name__ == "__main__":
    main()
