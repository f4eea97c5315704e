#!/usr/bin/env python
"""Benchmark: ELBO + gradient source-pixel evaluations per second on one synthetic
SDSS-shaped field (5 bands x 2048 x 1489 px, 500 sources), FP32 per-pixel arithmetic
with FP64 accumulation, next to the plain FP64 path, the end-to-end host-pointer call
and the FP64 CPU oracle.

One step = one ELBO + gradient evaluation of every source of the field (the patch
tables and KL terms, every item's mixture values and derivatives with its neighbours'
E/Var at multiply covered pixels, log-likelihood, adjoint and chain rule, then the
per-source epilogues and the total), i.e. one source-pixel evaluation per (source,
active pixel) pair.  Inputs are resident on the device; L2 is flushed (256 MiB write)
between timed steps, outside the timed events.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
  python bench.py --step-only ...    the FP32 step alone (the profiling command)
  python bench.py --fit-only ...     the Newton fit alone (the fit's profiling command)
  python bench.py --workload N ...   another workload as the step (see --help)
Multi-GPU (torchrun): every rank evaluates its own field (weak scaling, no collective
on the data path); timing is the max over ranks.

Besides the step (`value`, `e2e`, `fp64_path` with its FP64 roofline) the JSON line
carries: `roofline` (the item kernel's achieved FLOP rate against the FP32 peak derived
from unit counts and clock, its DRAM bytes per launch imported from an ncu capture,
every stage's CUDA-event time as the call runs them and serialised on one stream, and
`step`: the whole step against its plain-ALU bound); `cpu_baseline` (the FP64 oracle on
all host cores and on one); `hessian` (with its FLOP count, roofline, the Hessian
pass's own roofline, cost relative to ELBO + gradient and the CUDA-event time of each
of its stages), `fit` (with the FP32 sweeps alone, `fp32_only`, and fit quality),
`fit_schedules`, `catalog`, `workloads` (the crowded region, the sweep field and the
multi-epoch region) and `tasks` legs; `clocks` sampled around and during the timed
region; `gpu_launches`.  `--impl reference` times the oracle instead (rank 0 only) on a
bounded sample of the same field.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1801_10277_gb300 import synth  # noqa: E402

FLUSH_BYTES = 256 << 20
SM_COUNT = 152
# DRAM bytes (read + write) per launch of the item kernel on the one-field workload, from one
# ncu capture (profiles/k_items_field_500src.md); emptied whenever the kernel changes after
# the capture.
DRAM_BYTES_PER_LAUNCH = {"items": 26240256}
DRAM_BYTES_SOURCE = "ncu capture of one k_items launch, profiles/k_items_field_500src.md (imported, not measured here)"
FP32_LANES = 128
XU_LANES = 16   # MUFU ex2 results per SM per clock
SM_MHZ_MAX = 2070.0


def step_bound(npsf, n_exp, n_dev, value, other_per_sp=0.0):
    """The whole step's plain-ALU bound in source-pixel evals/s: the FP32 pipe at its
    peak doing the item kernel's algorithmic FLOP for every source-pixel (and the other
    sources' values at multiply covered pixels, other_per_sp per source-pixel), or the
    ex2 unit doing its exps (one per mixture component), whichever is slower; and value's
    fraction of it."""
    per_sp = items_flops_per_source_pixel(npsf, n_exp, n_dev) + other_per_sp * other_eval_flops(npsf, n_exp, n_dev)
    fp32 = SM_COUNT * FP32_LANES * 2 * SM_MHZ_MAX * 1e6 / per_sp
    xu = SM_COUNT * XU_LANES * SM_MHZ_MAX * 1e6 / (npsf * (1 + n_exp + n_dev) * (1 + other_per_sp))
    bound = min(fp32, xu)
    return {"bound": "alu", "evals_per_s_fp32_pipe": fp32, "evals_per_s_ex2": xu,
            "evals_per_s_bound": bound, "value": value, "frac": value / bound,
            "flop_per_source_pixel": per_sp}


def items_flops_per_source_pixel(npsf, n_exp, n_dev):
    """Algorithmic FP32 operations (FMA = 2) of the item kernel per source-pixel of the
    item's own patch (value + gradient), counted from the formulas it evaluates in the
    frame whitening each PSF component: per PSF component the offset, whitened
    coordinates and their squares (11), the star component (exponent 2, value 2, mean
    derivative 11), each galaxy component (exponent 4, value 1, the two mean and three
    shape sums 14) and the map back through T (41); per pixel the profile value and
    e_dev derivative (4), E_s and Var_s (27), E (1), the likelihood (8), its two weights
    (9) and the 12 y-gradients (65)."""
    nprof = n_exp + n_dev
    return npsf * (67 + 19 * nprof) + 114


def fp64_path_flops_per_source_pixel(npsf, n_exp, n_dev):
    """Algorithmic operations of the FP64 path per source-pixel (FMA = 2), counted from the
    formulas of its two passes: the map pass (per PSF component the offset and its
    products 5, the star 8, each galaxy component exponent 6 and weighted sum 2; per pixel
    E_s and Var_s 30) and the adjoint, which recomputes the mixture with its derivatives
    (per PSF component 5 + 18, each galaxy component 33; per pixel the likelihood weights
    and the 12 y-gradients 55).  The gather's ~10 operations per multiply covered pixel
    are left out."""
    nprof = n_exp + n_dev
    return npsf * (5 + 8 + 8 * nprof) + 30 + npsf * (5 + 18 + 33 * nprof) + 55


def hess_pass_flops_per_source_pixel(npsf, n_exp, n_dev):
    """Algorithmic operations of the FP32 Hessian pass (`k_hess<float>`) per source-pixel
    (FMA = 2); it evaluates the galaxy mixture in the frame whitening each PSF component.
    Per PSF component: the offset and its products (5), the star component with its first
    and second derivatives (31), the whitened coordinates and their squares (8), each
    galaxy component's exponent and value (5) and its 35 weighted sums (70), and the sums'
    map back to the pixel frame (329: the z-monomials, the whitened gradient and Hessian
    blocks, their transforms through T and K); per pixel the 78 packed y-Hessian entries,
    the gradient and the likelihood weights (600)."""
    nprof = n_exp + n_dev
    return npsf * (5 + 31 + 8 + 329 + 75 * nprof) + 600


def hess_flops_per_source_pixel(npsf, n_exp, n_dev):
    """The whole FP32 Hessian evaluation per source-pixel: the map pass (as in
    fp64_path_flops_per_source_pixel) and the Hessian pass."""
    nprof = n_exp + n_dev
    return npsf * (5 + 8 + 8 * nprof) + 30 + hess_pass_flops_per_source_pixel(npsf, n_exp, n_dev)


def hess64_flops_per_source_pixel(npsf, n_exp, n_dev):
    """The same for the FP64 Hessian path, which evaluates the mixture's first and second
    derivatives component by component in the pixel frame (per PSF component 20 + 42, each
    galaxy component 140; per pixel 600)."""
    nprof = n_exp + n_dev
    return npsf * (5 + 8 + 8 * nprof) + 30 + npsf * (20 + 42 + 140 * nprof) + 600


# FP64 peak, derived: 152 SMs x 2 FP64 FMA lanes per clock (the FP64 pipe's width on this
# part) x 2 FLOP x the 2070 MHz maximum clock
FP64_LANES = 2


def hessian_summary(n_sp, ws, npsf, n_exp, n_dev, ms32, ms64, stage_us, elbo_grad_value):
    """The `hessian` leg of the JSON line from its measurements: ms32 / ms64 the FP32 and
    FP64 evaluations' CUDA-event milliseconds, stage_us the FP32 evaluation's stages (µs
    per launch), n_sp the source-pixels per rank, ws ranks.  `roofline` is the whole
    evaluation against the FP32 peak (and the FP64 path against the FP64 peak);
    `roofline.kernel` is the Hessian pass alone (its stage time), null if the stage is
    missing."""
    peak_fp32 = SM_COUNT * FP32_LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12
    peak_fp64 = SM_COUNT * FP64_LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12
    hflop = hess_flops_per_source_pixel(npsf, n_exp, n_dev)
    h64flop = hess64_flops_per_source_pixel(npsf, n_exp, n_dev)
    pflop = hess_pass_flops_per_source_pixel(npsf, n_exp, n_dev)
    h32 = n_sp * ws / (ms32 / 1000.0)
    h64 = n_sp * ws / (ms64 / 1000.0)
    k_us = stage_us.get("hess_adjoint")
    kernel = None
    if k_us:
        k_ach = pflop * n_sp / (k_us * 1e-6) / 1e12
        kernel = {"name": "k_hess<float>", "us": k_us, "flop_per_source_pixel": pflop,
                  "achieved": k_ach, "frac": k_ach / peak_fp32}
    return {"value": h32, "unit": "source-pixel evals/s",
            "ms_per_step": ms32, "fp64_value": h64,
            "fp64_ms_per_step": ms64,
            "what": "ELBO + gradient + 44x44 Hessian of every source",
            "cost_vs_elbo_grad": elbo_grad_value / h32,
            "stage_us": stage_us,
            "roofline": {"bound": "alu", "flop_per_source_pixel": hflop,
                         "achieved": hflop * h32 / ws / 1e12, "peak": peak_fp32, "unit": "TFLOP/s",
                         "frac": hflop * h32 / ws / 1e12 / peak_fp32,
                         "peak_source": "FP32: 152 SM x 128 lanes x 2 x 2070 MHz (unit counts, max clock)",
                         "kernel": kernel,
                         "fp64": {"flop_per_source_pixel": h64flop,
                                  "achieved": h64flop * h64 / ws / 1e12, "peak": peak_fp64,
                                  "frac": h64flop * h64 / ws / 1e12 / peak_fp64,
                                  "peak_source": "152 SM x 2 FP64 lanes x 2 x 2070 MHz (derived)"}}}


def other_eval_flops(npsf, n_exp, n_dev):
    """FP32 operations of one other covering source's E and Var at a multiply covered
    pixel: per PSF component the coordinates (11), star exponent and value (4), each
    galaxy component's exponent and value (5), the component's sums (6); then the profile
    value (3), E_s and Var_s (27) and the two additions (2)."""
    nprof = n_exp + n_dev
    return npsf * (21 + 5 * nprof) + 32


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, idx):
        self.idx = idx
        self.p = None

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def once(self):
        """One sample, taken immediately (a short timed region may end between the
        periodic samples)."""
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            return r.stdout if r.returncode == 0 else ""
        except Exception:
            return ""

    def __enter__(self):
        self.first = self.once()
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
        self.out = (self.first or "") + (self.out or "") + self.once()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_init(backend="nccl"):
    """(rank, world size, torch.distributed or None) from the torchrun environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    dist.init_process_group(backend)
    return dist.get_rank(), ws, dist


def rank_field_seed(rank):
    """Weak scaling: every rank evaluates its own synthetic field (the one-field
    recipe with its own seed); no data crosses ranks."""
    return 2027 + rank


def max_over_ranks(x, dist, device):
    """The slowest rank's value (a time), identical on every rank."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_rate(prob, min_seconds=10.0, max_reps=200, threads=None):
    """FP64 CPU oracle ELBO + gradient over the whole of prob, repeated until
    min_seconds of work, on all host cores or on `threads` of them; returns
    (source-pixel evals/s, cores, reps, seconds)."""
    from oracle.oracle import Oracle, num_threads, set_threads
    prev = num_threads()
    if threads:
        set_threads(threads)
    try:
        cores = num_threads()
        orc = Oracle(prob)
        reps, t0 = 0, time.perf_counter()
        while True:
            orc.elbo(prob.theta)
            orc.derivs(prob.theta)
            reps += 1
            el = time.perf_counter() - t0
            if el >= min_seconds or reps >= max_reps:
                break
    finally:
        set_threads(prev)
    return prob.source_pixels() * reps / el, cores, reps, el


def reference_sample(prob, steps, warmup, budget_s=120.0):
    """The bounded sample one reference step evaluates: every stride-th source of the
    field (their patches, the images unchanged), stride chosen from one timed
    whole-field evaluation so that warmup + steps evaluations take about budget_s."""
    from oracle.oracle import Oracle
    orc = Oracle(prob)
    t0 = time.perf_counter()
    orc.elbo(prob.theta)
    orc.derivs(prob.theta)
    t_full = time.perf_counter() - t0
    per_step = budget_s / max(1, steps + warmup)
    frac = min(1.0, per_step / max(t_full, 1e-9))
    n = max(1, int(prob.n_src * frac))
    stride = max(1, prob.n_src // n)
    idx = np.arange(0, prob.n_src, stride)
    return (prob if stride == 1 else synth.subset(prob, idx)), stride


def reference_arm(args, rank, ws):
    """--impl reference: the oracle as it stands on the host cores (rank 0 only), each
    step one ELBO + gradient evaluation of a bounded sample of the field."""
    if rank != 0:
        return
    from oracle.oracle import Oracle, num_threads
    prob = synth.config(1)
    sample, stride = reference_sample(prob, args.steps, args.warmup)
    orc = Oracle(sample)
    for _ in range(args.warmup):
        orc.elbo(sample.theta)
        orc.derivs(sample.theta)
    t_steps = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        orc.elbo(sample.theta)
        orc.derivs(sample.theta)
        t_steps.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(t_steps) / len(t_steps)
    n_sp = sample.source_pixels()
    val = n_sp / (ms / 1000.0)
    which = "the whole field" if stride == 1 else f"sources 0, {stride}, {2 * stride}, ... of the field"
    desc = (f"{which} ({sample.n_src} sources, {n_sp} source-pixels), one FP64 ELBO + "
            f"gradient evaluation per step")
    line = {
        "impl": "reference", "metric": "ELBO+grad source-pixel evals/s", "value": val,
        "unit": "source-pixel evals/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": prob.name, "sources": prob.n_src,
                   "source_pixels": prob.source_pixels(), "images": len(prob.images),
                   "image": "x".join(str(v) for v in prob.images[0].pixels.shape[::-1]),
                   "precision": "fp64", "l2": "not applicable (host)", "tuning": None,
                   "parallelism": "single", "sample": desc,
                   "hardware": "host cores of rank 0; no GPU"},
        "cpu_baseline": {"value": val, "unit": "source-pixel evals/s", "cores": num_threads(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": "source-pixel evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def model_image_fit(cel, prob, P, seed=7):
    import copy
    truth = prob.truth.copy()
    star = truth[:, synth.I_A] >= 0.5
    truth[:, synth.I_A] = np.where(star, 0.995, 0.005)
    truth[:, synth.I_A + 1] = 1.0 - truth[:, synth.I_A]
    E, _ = P.render(truth)
    rng = np.random.default_rng(seed)
    pm = copy.copy(prob)
    pm.images = [copy.copy(im) for im in prob.images]
    for im, e in zip(pm.images, E):
        im.pixels = rng.poisson(e).astype(np.float32)
    Pm = cel.Problem(pm)
    t0 = time.perf_counter()
    th_fit, iters, fst, _ = Pm.fit(prob.theta, precision=cel.FP32, max_sweeps=3)
    secs = time.perf_counter() - t0
    cat_true = Pm.catalog(truth)
    cat_fit = Pm.catalog(th_fit)
    bright = np.exp(truth[:, synth.I_R1]) >= 10.0   # r flux >= 10 nmgy
    out = {"start": Pm.catalog_score(Pm.catalog(prob.theta), cat_true),
           "fitted": Pm.catalog_score(cat_fit, cat_true),
           "fitted_bright": Pm.catalog_score(cat_fit[bright], cat_true[bright]),
           "seconds": secs, "converged": int((fst == 0).sum()),
           "data": f"Poisson counts around the model's expected image at the truth (seed {seed})"}
    Pm.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=20)
    ap.add_argument("--hess-steps", type=int, default=20)
    ap.add_argument("--no-fit", action="store_true")
    ap.add_argument("--no-schedules", action="store_true",
                    help="skip the colour vs Cyclades convergence-per-sweep leg")
    ap.add_argument("--schedule-sweeps", type=int, default=4)
    ap.add_argument("--no-tasks", action="store_true", help="skip the region-task leg")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workloads' legs (crowded region, sweep field, multi-epoch region)")
    ap.add_argument("--fit-only", action="store_true",
                    help="time the Newton fit of the workload alone (FP32 sweeps, FP64 polish)")
    ap.add_argument("--step-only", action="store_true",
                    help="run the FP32 value + gradient step alone (warm-up and timed steps, no other "
                         "leg): the profiling command for the step's kernels")
    ap.add_argument("--workload", type=int, default=1, choices=[1, 2, 3, 4, 5, 6],
                    help="1 one field (the benchmark), 2 crowded region, 3 multi-epoch region, "
                         "4 sweep field, 5 deep stack (480 images per source), 6 the whole 200,000-source "
                         "sweep (64 fields); the JSON line names it")
    ap.add_argument("--tuning", default=None,
                    help="contrib,items codes to use instead of autotuning (e.g. 2,3)")
    args = ap.parse_args()
    if args.impl == "reference":
        # rank 0 alone times the oracle; no process group is needed for that
        reference_arm(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, ws, dist = dist_init()
    import torch
    from paper_1801_10277_gb300 import celeste as cel
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    if args.workload == 1:
        prob = synth.config(1, seed=rank_field_seed(rank))
    else:
        prob = synth.config(args.workload)
    P = cel.Problem(prob)
    n_sp = P.source_pixels
    if args.tuning:
        tuning = tuple(int(v) for v in args.tuning.split(","))
        P.set_tuning(*tuning)
    else:
        tuning = P.autotune(prob.theta)
    if args.fit_only:
        # the Newton fit alone (the profiling command for the fit's kernels)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, iters, fst, el = P.fit(prob.theta, precision=cel.FP32, max_sweeps=3)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        if rank == 0:
            print(json.dumps({"metric": "Newton iterations/s", "value": float(iters.sum()) / secs,
                              "unit": "iterations/s", "seconds": secs, "newton_iterations": int(iters.sum()),
                              "converged": int((fst == 0).sum()), "elbo": el,
                              "config": {"workload": prob.name, "sources": prob.n_src}}), flush=True)
        return
    dev = torch.device("cuda", local_rank)
    theta = torch.tensor(prob.theta, dtype=torch.float64, device=dev)
    if args.step_only:
        # the FP32 step alone, for a profiler's launch list or a capture of one kernel
        tot = torch.zeros(1, dtype=torch.float64, device=dev)
        loc = torch.zeros(prob.n_src, dtype=torch.float64, device=dev)
        grad = torch.zeros(prob.n_src, 44, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            P.elbo_grad_device(theta, tot, loc, grad, precision=cel.FP32)
        torch.cuda.synchronize()
        if P.device_status() != 0:
            raise RuntimeError("device-side parameter check failed")
        if rank == 0:
            print(json.dumps({"step_only": True, "steps": args.warmup + args.steps, "elbo": float(tot.item()),
                              "tuning": list(tuning), "config": {"workload": prob.name, "sources": prob.n_src}}),
                  flush=True)
        return
    tot = torch.zeros(1, dtype=torch.float64, device=dev)
    loc = torch.zeros(prob.n_src, dtype=torch.float64, device=dev)
    grad = torch.zeros(prob.n_src, 44, dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(prec):
        P.elbo_grad_device(theta, tot, loc, grad, precision=prec)

    def timed_loop(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step(prec)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        return max_over_ranks(ms, dist, dev)

    with Clocks(local_rank) as clk:
        ms32 = timed_loop(cel.FP32, args.steps, args.warmup)
    if P.device_status() != 0:
        raise RuntimeError("device-side parameter check failed")
    value = n_sp * ws / (ms32 / 1000.0)
    ms64 = timed_loop(cel.FP64, args.fp64_steps, 1)
    value64 = n_sp * ws / (ms64 / 1000.0)

    # per-kernel durations (CUDA events on each kernel's launch stream), FP32 path
    P.profile(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step(cel.FP32)
    torch.cuda.synchronize()
    prof = P.profile_read()
    # the same stages serialised on one stream: the shares a serialised launch list shows
    P.profile(True, serial=True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        step(cel.FP32)
    torch.cuda.synchronize()
    prof_serial = P.profile_read()
    P.profile(False)
    tot_serial = sum(v[0] for v in prof_serial.values())
    launches_per_step = sum(v[1] for v in prof.values()) / args.steps
    kernel_us = {k: 1000.0 * v[0] / max(1, v[1]) for k, v in prof.items()}
    tot_ms = sum(v[0] for v in prof.values())
    npsf = prob.images[0].psf.shape[0]
    ne, nd = prob.exp_mix.shape[0], prob.dev_mix.shape[0]
    split = P.stats()
    # algorithmic FP32 FLOP of one launch of the item kernel: every source-pixel of its own
    # patch, plus the other covering sources' E and Var at multiply covered pixels
    work = {"items": items_flops_per_source_pixel(npsf, ne, nd) * n_sp
                     + other_eval_flops(npsf, ne, nd) * split["other_evals"]}
    achieved_k = {k: work[k] / (kernel_us[k] * 1e-6) / 1e12 for k in work if kernel_us.get(k, 0) > 0}
    dom = "items"
    clocks = clk.summary()
    peak_fp32 = SM_COUNT * FP32_LANES * 2 * 2070e6 / 1e12
    achieved = achieved_k[dom]
    traffic = DRAM_BYTES_PER_LAUNCH.get(dom) if args.workload == 1 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                "frac": achieved / peak_fp32, "traffic": traffic,
                "traffic_source": DRAM_BYTES_SOURCE if traffic is not None else None,
                "kernel": "items: k_items, the FP32 value + gradient pass over every item (the tables "
                          "and KL terms, and the per-source epilogues, are the stages 'tables' and 'finish')",
                "flop_per_launch": work[dom],
                "flop_per_source_pixel": items_flops_per_source_pixel(npsf, ne, nd),
                "other_evals": split["other_evals"], "flop_per_other_eval": other_eval_flops(npsf, ne, nd),
                "peak_source": "152 SM x 128 FP32 lanes x 2 x 2070 MHz (unit counts and max clock)",
                "kernel_us": kernel_us, "kernel_tflops": achieved_k,
                "kernel_share": {k: v[0] / tot_ms for k, v in prof.items()},
                "step": step_bound(npsf, ne, nd, value / ws, split["other_evals"] / n_sp),   # per GPU
                "kernel_us_serialised": {k: 1000.0 * v[0] / max(1, v[1]) for k, v in prof_serial.items()},
                "kernel_share_serialised": {k: v[0] / tot_serial for k, v in prof_serial.items()},
                "work_split": split}

    # Hessian (value + gradient + per-source 44 x 44 Hessian), FP32 and FP64 pixel paths
    hes = torch.zeros(prob.n_src, 44, 44, dtype=torch.float64, device=dev)

    def hess_loop(prec, steps):
        P.hess_device(theta, loc, grad, hes, precision=prec)
        torch.cuda.synchronize()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            P.hess_device(theta, loc, grad, hes, precision=prec)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / steps

    hms32 = hess_loop(cel.FP32, args.hess_steps)
    hms64 = hess_loop(cel.FP64, max(1, args.hess_steps // 10))
    # the FP32 Hessian evaluation's stages (CUDA events on each stage's launch stream)
    P.profile(True)
    for _ in range(args.hess_steps):
        flush.fill_(1.0)
        P.hess_device(theta, loc, grad, hes, precision=cel.FP32)
    torch.cuda.synchronize()
    hprof = P.profile_read()
    P.profile(False)
    hstage_us = {k: 1000.0 * v[0] / max(1, v[1]) for k, v in hprof.items()}
    hessian = hessian_summary(n_sp, ws, npsf, ne, nd, hms32, hms64, hstage_us, value)
    f64flop = fp64_path_flops_per_source_pixel(npsf, ne, nd)
    peak_fp64 = SM_COUNT * FP64_LANES * 2 * SM_MHZ_MAX * 1e6 / 1e12

    # end to end through the host-pointer C ABI (pinned buffers, copies inside)
    pin_th = torch.tensor(prob.theta, dtype=torch.float64).pin_memory()
    pin_tot = torch.zeros(1, dtype=torch.float64).pin_memory()
    pin_loc = torch.zeros(prob.n_src, dtype=torch.float64).pin_memory()
    pin_g = torch.zeros(prob.n_src, 44, dtype=torch.float64).pin_memory()
    import ctypes as C

    def host_step():
        st = P.L.celeste_elbo_grad(P.h, C.c_void_p(pin_th.data_ptr()), cel.FP32,
                                   C.c_void_p(pin_tot.data_ptr()), C.c_void_p(pin_loc.data_ptr()),
                                   C.c_void_p(pin_g.data_ptr()))
        cel._check(st)

    for _ in range(args.warmup):
        host_step()
    t_e2e = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        host_step()
        t_e2e.append(time.perf_counter() - t0)
    e2e_ms = 1000.0 * sum(t_e2e) / len(t_e2e)
    e2e_ms = max_over_ranks(e2e_ms, dist, dev)
    e2e = {"value": n_sp * ws / (e2e_ms / 1000.0), "unit": "source-pixel evals/s",
           "h2d_bytes_per_step": int(pin_th.numel() * 8),
           "d2h_bytes_per_step": int((pin_tot.numel() + pin_loc.numel() + pin_g.numel()) * 8),
           "ms_per_step": e2e_ms}

    # Newton fit of the whole field from the perturbed start (trust region per source,
    # colour by colour, FP32 sweeps polished by FP64 sweeps); host wall clock
    fit = None
    if not args.no_fit:
        el_start = P.elbo(prob.theta, precision=cel.FP64)[0]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th_fit, iters, fst, el_fit = P.fit(prob.theta, precision=cel.FP32, max_sweeps=3)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        fit = {"newton_iterations_per_s": float(iters.sum()) / secs, "seconds": secs,
               "newton_iterations": int(iters.sum()), "sources": prob.n_src,
               "elbo_start": el_start, "elbo_end": el_fit,
               "converged": int((fst == 0).sum()),
               "options": "FP32 pixels, FP64 refinement, <= 3 sweeps, <= 50 iterations per source"}
        # the FP32 sweeps alone (no FP64 polish): the fit targets hold for them too
        # (tests/test_gpu_fit.py), so this is the FP32 path's own fit time
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it32, fst32, el32 = P.fit(prob.theta, precision=cel.FP32, refine_fp64=0, max_sweeps=3)
        torch.cuda.synchronize()
        s32 = time.perf_counter() - t0
        fit["fp32_only"] = {"seconds": s32, "newton_iterations": int(it32.sum()),
                            "newton_iterations_per_s": float(it32.sum()) / s32,
                            "converged": int((fst32 == 0).sum()), "elbo_end": el32,
                            "options": "FP32 pixels, FP64 accumulation, no FP64 polish, <= 3 sweeps"}
        # fit quality against the generator's truth (Table II's error summary; the images
        # are isotropic blobs, so galaxy shape truth is not in the pixels)
        cat_true = P.catalog(prob.truth)
        fit["quality"] = {"start": P.catalog_score(P.catalog(prob.theta), cat_true),
                          "fitted": P.catalog_score(P.catalog(th_fit), cat_true)}
        # the same fit on images drawn from the model itself: Poisson counts around the
        # expected image at the truth (types as q(star) = 0.995 / 0.005)
        fit["quality_model_images"] = model_image_fit(cel, prob, P)

    # catalog rows with posterior uncertainty for every source (one kernel)
    d_th = torch.tensor(prob.theta, dtype=torch.float64, device="cuda")
    d_cat = torch.empty(prob.n_src, cel.CAT_NFIELD, dtype=torch.float64, device="cuda")
    for _ in range(5):
        P.catalog_device(d_th, d_cat)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(100):
        P.catalog_device(d_th, d_cat)
    ev1.record()
    torch.cuda.synchronize()
    cat_ms = ev0.elapsed_time(ev1) / 100
    catalog = {"sources_per_s": prob.n_src / (cat_ms / 1000.0), "ms_per_call": cat_ms,
               "fields": cel.CAT_NFIELD}

    # convergence per sweep of the two conflict-free schedules (Section IV-D): greedy
    # colouring vs Cyclades samples (sweep k's order drawn in the library from seed k);
    # one sweep per call from the previous sweep's result, FP32 pixels, no polish; the
    # ELBO after each sweep in FP64, outside the timed calls
    schedules = None
    if not args.no_fit and not args.no_schedules:
        schedules = {}
        for name, kw in (("colour", {}),
                         ("cyclades_64", dict(schedule="cyclades", sample_size=64)),
                         ("cyclades_all", dict(schedule="cyclades", sample_size=prob.n_src))):
            th = prob.theta.copy()
            elbos, secs_l, iters_l = [], [], []
            for k in range(args.schedule_sweeps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                th, iters, _, _ = P.fit(th, precision=cel.FP32, refine_fp64=0, max_sweeps=1,
                                        seed=k, **kw)
                torch.cuda.synchronize()
                secs_l.append(time.perf_counter() - t0)
                iters_l.append(int(iters.sum()))
                elbos.append(P.elbo(th, precision=cel.FP64)[0])
            entry = {"elbo_after_sweep": elbos, "seconds_per_sweep": secs_l,
                     "newton_iterations_per_sweep": iters_l}
            if kw:   # batches per sweep, mean over four random orders
                rng = np.random.default_rng(0)
                entry["batches_per_sweep"] = float(np.mean([cel.cyclades_batches(
                    prob.nbr_offsets, prob.nbrs, rng.permutation(prob.n_src).astype(np.int32),
                    kw["sample_size"])[2] for _ in range(4)]))
            schedules[name] = entry
        schedules["elbo_start"] = P.elbo(prob.theta, precision=cel.FP64)[0]

    # region tasks (Section IV-A) on one GPU: one global fit against one and two stages of
    # tasks (regions of about 1/16 of the work; the second stage shifted by half a
    # region), FP32 sweeps polished in FP64; total ELBO after each and host wall time
    # The other workloads, each timed like the headline (device-resident inputs, L2
    # flushed between steps) with the headline's variant codes, and its item kernel's
    # share of the FP32 peak.  Single-GPU runs only (every rank would repeat them).
    workloads = None
    if not args.no_workloads and args.workload == 1 and ws == 1:
        workloads = {}
        for wc, wsteps in ((2, args.steps), (4, max(3, args.steps // 4)), (3, 3)):
            wp = synth.config(wc)
            WP = cel.Problem(wp)
            WP.set_tuning(*tuning)
            w_th = torch.tensor(wp.theta, dtype=torch.float64, device=dev)
            w_tot = torch.zeros(1, dtype=torch.float64, device=dev)
            w_loc = torch.zeros(wp.n_src, dtype=torch.float64, device=dev)
            w_gr = torch.zeros(wp.n_src, 44, dtype=torch.float64, device=dev)

            def wstep():
                WP.elbo_grad_device(w_th, w_tot, w_loc, w_gr, precision=cel.FP32)

            for _ in range(2):
                wstep()
            torch.cuda.synchronize()
            evs = []
            for _ in range(wsteps):
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                wstep()
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
            wms = sum(a.elapsed_time(b) for a, b in evs) / wsteps
            WP.profile(True)
            for _ in range(wsteps):
                flush.fill_(1.0)
                wstep()
            torch.cuda.synchronize()
            wprof = WP.profile_read()
            WP.profile(False)
            w_sp = WP.source_pixels
            wsplit = WP.stats()
            w_npsf = wp.images[0].psf.shape[0]
            wwork = (items_flops_per_source_pixel(w_npsf, ne, nd) * w_sp
                     + other_eval_flops(w_npsf, ne, nd) * wsplit["other_evals"])
            w_items_us = 1000.0 * wprof["items"][0] / max(1, wprof["items"][1])
            w_val = w_sp / (wms / 1000.0)
            w_ach = wwork / (w_items_us * 1e-6) / 1e12
            workloads[wp.name] = {
                "value": w_val, "unit": "source-pixel evals/s", "ms_per_step": wms, "steps": wsteps,
                "sources": wp.n_src, "source_pixels": w_sp,
                "roofline": {"bound": "alu", "kernel": "items", "achieved": w_ach, "peak": peak_fp32,
                             "unit": "TFLOP/s", "frac": w_ach / peak_fp32, "flop_per_launch": wwork,
                             "kernel_us": {k: 1000.0 * v[0] / max(1, v[1]) for k, v in wprof.items()}},
                "step": step_bound(w_npsf, ne, nd, w_val, wsplit["other_evals"] / w_sp)}
            WP.close()
            del WP, wp, w_th, w_loc, w_gr
            torch.cuda.empty_cache()

    tasks = None
    if not args.no_fit and not args.no_tasks:
        npx = np.zeros(prob.n_src)
        np.add.at(npx, np.repeat(np.arange(prob.n_src), np.diff(prob.patch_offsets)),
                  prob.patches[:, 3].astype(np.float64) * prob.patches[:, 4])
        pos = prob.theta[:, 0:2]
        t1, n1 = cel.make_tasks(pos, npx, npx.sum() / 16)
        span = pos.max(axis=0) - pos.min(axis=0)
        shift = 0.5 * span / 4.0   # about half a region of a 4 x 4 cut
        t2, n2 = cel.make_tasks(pos, npx, npx.sum() / 16, shift)
        kw = dict(precision=cel.FP32, max_sweeps=3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, _, el_g = P.fit(prob.theta, **kw)
        torch.cuda.synchronize()
        sec_g = time.perf_counter() - t0
        t0 = time.perf_counter()
        th1, _, _, el_1 = P.fit_tasks(prob.theta, t1, **kw)
        sec_1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        _, _, _, el_2 = P.fit_tasks(th1, t2, **kw)
        sec_2 = time.perf_counter() - t0
        tasks = {"tasks_per_stage": [n1, n2], "shift": shift.tolist(),
                 "elbo_start": P.elbo(prob.theta, precision=cel.FP64)[0],
                 "global_fit": {"elbo": el_g, "seconds": sec_g},
                 "stage1": {"elbo": el_1, "seconds": sec_1},
                 "stage2": {"elbo": el_2, "seconds": sec_2}}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, reps, secs = oracle_rate(prob)
        cpu = {"value": rate, "unit": "source-pixel evals/s", "cores": cores, "kind": "oracle",
               "sample": f"whole field ({n_sp} source-pixels) ELBO + gradient x {reps} "
                         f"({secs:.1f} s)"}
        # the same on one core, on every 10th source of the field
        sub = synth.subset(prob, np.arange(0, prob.n_src, 10)) if prob.n_src >= 100 else prob
        rate1, _, reps1, secs1 = oracle_rate(sub, min_seconds=5.0, threads=1)
        cpu["one_core"] = {"value": rate1, "unit": "source-pixel evals/s", "cores": 1,
                           "sample": f"every 10th source ({sub.source_pixels()} source-pixels) "
                                     f"ELBO + gradient x {reps1} ({secs1:.1f} s)"}
    if rank == 0:
        line = {
            "metric": "ELBO+grad source-pixel evals/s", "value": value,
            "unit": "source-pixel evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": prob.name, "sources": prob.n_src, "source_pixels": n_sp,
                       "images": len(prob.images),
                       "image": "x".join(str(v) for v in prob.images[0].pixels.shape[::-1]),
                       "precision": "fp32 pixels, fp64 accumulation",
                       "l2": "flushed between steps (256 MiB write)",
                       "tuning": dict(zip(("contrib", "items"), tuning)),
                       "parallelism": f"replica{ws}" if ws > 1 else "single"},
            "fp64_path": {"value": value64, "unit": "source-pixel evals/s", "ms_per_step": ms64,
                          "speedup_fp32_over_fp64": value / value64,
                          "roofline": {"bound": "alu", "flop_per_source_pixel": f64flop,
                                       "achieved": f64flop * value64 / ws / 1e12, "peak": peak_fp64,
                                       "unit": "TFLOP/s", "frac": f64flop * value64 / ws / 1e12 / peak_fp64,
                                       "peak_source": "152 SM x 2 FP64 lanes x 2 x 2070 MHz (derived)"}},
            "workloads": workloads,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "hessian": hessian, "fit": fit, "fit_schedules": schedules, "catalog": catalog, "tasks": tasks,
            "gpu_launches": int(round(launches_per_step * args.steps)),
        }
        print(json.dumps(line), flush=True)
    P.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
