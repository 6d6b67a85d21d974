#!/usr/bin/env python
"""Benchmark of the binned Poisson -lnL + adjoint (arXiv:1805.11125 multivariate fit model).

Workload: the multivariate model (K = 15 species, TFC-vetoed and TFC-tagged spectra of 900
1-npe bins over 100-1000 npe, a 60-bin radial and a 50-bin pulse-shape histogram, 22
parameters, 2e6 events), synthetic and seeded.  One step evaluates -lnL and its gradient
at a batch of parameter points (theta_true * (1 + 0.02 z)) through the C ABI
(bx_nll_batch, FP32 mixed precision, device pointers).  The FP64 GPU form is timed beside
it, the oracle (plain FP64 C on the host cores) gives the CPU baseline.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU with its own
batch (weak scaling; the likelihood of one dataset does not need a collective).
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "-lnL+grad evals/s & full-fit wall time, mixed vs FP64 GPU at |Δ(-2lnL)|≤1e-3"
WORKLOAD = ("multivariate spectral fit: K=15 species on a 2000-point 0-3 MeV grid, TFC-vetoed + TFC-tagged "
            "900x1 npe (100-1000 npe), radial 60, pulse-shape 50, 22 parameters, 2e6 events, pile-up L=400")
# FP32 operations per in-band response entry of the forward kernel, counted from the source
# (bx_resp.cuh resp_shape32 44, two Kahan row sums 8, column sum 2)
FWD_OPS_PER_ENTRY = 54
# adjoint kernel per entry of a run of 16 rows (bx_resp.cuh adj_run): recurrence 7, outer-node
# products 2, basis sums 19 (AdjSums::add), weight 3, plus the exact start of the run (58) / 16
BWD_OPS_PER_ENTRY = 35
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes (read + write) per evaluation item of the two candidate dominant kernels, from one
# ncu capture of the multivariate model at 512 items (--set full, one launch each); the traffic
# scales with the items of a launch.
TRAFFIC_PER_ITEM = {"k_fwd_f32": (45.5e6 + 2.85e6) / 512, "k_bwd_f32": (96.9e6 + 3.14e6) / 512}


def job_throughput(local_ms: float, items_per_rank: int, steps: int, ws: int, device=None):
    """Whole-job evaluations/s of a weak-scaling replica run: every rank evaluated
    items_per_rank x steps items in local_ms; the job took the slowest rank's time (MAX over
    ranks; needs an initialised process group when ws > 1).  Returns (value, max_ms)."""
    max_ms = float(local_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([max_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_ms = float(t.item())
    return ws * items_per_rank * steps / (max_ms / 1e3), max_ms


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if len(r) > 5 + j and r[5 + j] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def make_dataset(bx, I, spec, seed=0):
    """Data drawn from the GPU model's own expected counts at theta_true."""
    dummy = spec.with_counts(np.zeros(spec.n_bins_total))
    m = bx.Model(dummy, precision=bx.BX_FP64)
    mu = m.expected(spec.theta_true)
    m.close()
    return spec.with_counts(I.poisson_counts(mu, seed))


def cpu_baseline(spec_name: str, seconds: float, seed: int = 0):
    """The oracle as it stands (FP64 C, dual-number gradient, OpenMP over output bins) on a
    bounded sample of the same workload: NLL+gradient at consecutive parameter points."""
    from oracle import oracle as O
    from paper_1805_11125_gb300 import inputs as I
    s = I.config(spec_name)
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), seed))
    pts = I.parameter_points(s.theta_true, 10000, rel=0.02, seed=11, free=s.default_free())
    om = O.OracleModel(s)
    O.nll(om, pts[0], grad=True)   # warm
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        O.nll(om, pts[n + 1], grad=True)
        n += 1
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} NLL+gradient evaluations of the multivariate model in {dt:.1f} s "
                      f"(one point at a time, OpenMP over output bins)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    cb = cpu_baseline("multivariate", max(args.cpu_seconds / max(args.steps, 1), 2.0))
    total_n, total_t = 0, 0.0
    # K timed steps of bounded samples, after W warm-up samples
    from oracle import oracle as O
    from paper_1805_11125_gb300 import inputs as I
    s = I.config("multivariate")
    s = s.with_counts(I.poisson_counts(O.expected(s, s.theta_true), 0))
    om = O.OracleModel(s)
    pts = I.parameter_points(s.theta_true, 4096, rel=0.02, seed=11, free=s.default_free())
    per_step = max(1, int(round(cb["value"] * args.cpu_seconds / max(args.steps, 1))))
    for w in range(args.warmup):
        O.nll(om, pts[w], grad=True)
    j = 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            O.nll(om, pts[j % len(pts)], grad=True)
            j += 1
        total_t += time.perf_counter() - t0
        total_n += per_step
    v = total_n / total_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "evals/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "global_batch": per_step,
                                              "l2": "n/a (host)"},
            "cpu_baseline": {"value": v, "unit": "evals/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": f"{per_step} NLL+gradient evaluations per step"},
            "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_1805_11125_gb300 import bx, inputs as I

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    spec = make_dataset(bx, I, I.config("multivariate"), seed=0)
    B = args.batch
    model = bx.Model(spec, precision=bx.BX_FP32, max_batch=B, stream=stream)
    P = model.P
    pts = I.parameter_points(spec.theta_true, B, rel=0.02, seed=100 + rank, free=spec.default_free())
    theta = torch.tensor(pts, dtype=torch.float64, device=dev)
    nll = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty((B, P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > 129 MB of L2

    def step():
        st = bx.lib().bx_nll_batch(model.h, B, None, bx._ptr(theta), bx._ptr(nll), bx._ptr(grad), 1)
        if st:
            raise bx.BxError(st, bx.lib().bx_last_error().decode())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    model.profile(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    stage_ms, n_evals, entries = model.profile(False)
    st = model.status()
    if st:
        raise bx.BxError(st, bx.lib().bx_last_error().decode())
    value, total_ms = job_throughput(sum(a.elapsed_time(b) for a, b in evs), B, args.steps, ws, dev)

    e2e, fp64_value, tc_value, fits, disc = None, None, None, None, None
    if not args.no_extras:
        e2e, fp64_value, tc_value = extras(bx, model, spec, pts, theta, stream, B, P, ws, args)
        fits = fit_times(bx, I, spec, stream)
        if args.toys > 0:
            fits["batched_toys"] = toy_fits(bx, I, args.toys, stream)
        disc = discrimination_leg(bx, I, stream, B=args.batch2d) if args.batch2d > 0 else None
        fits["quenched"] = variant_leg(bx, I, "quenched", QUENCHED, stream, B=args.batch) if args.quenched else None
        fits["sliced"] = variant_leg(bx, I, "sliced", SLICED, stream, B=args.batch) if args.sliced else None
        fits["joint_3d"] = (discrimination_leg(bx, I, stream, B=args.batch2d, name="joint", workload=JOINT,
                                               n_slices=120) if args.joint and args.batch2d > 0 else None)
    if rank != 0:
        return
    report(args, ws, B, total_ms, value, stage_ms, n_evals, entries, e2e, fp64_value, tc_value, clk, fits, disc)


def extras(bx, model, spec, pts, theta, stream, B, P, ws, args):
    import torch
    # end to end through the public call with host buffers (pinned), copies inside the region
    th_h = torch.tensor(pts, dtype=torch.float64).pin_memory()
    nll_h = torch.empty(B, dtype=torch.float64).pin_memory()
    grad_h = torch.empty((B, P), dtype=torch.float64).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    bx.lib().bx_nll_batch(model.h, B, None, th_h.data_ptr(), nll_h.data_ptr(), grad_h.data_ptr(), 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        s2 = bx.lib().bx_nll_batch(model.h, B, None, th_h.data_ptr(), nll_h.data_ptr(), grad_h.data_ptr(), 0)
        if s2:
            raise bx.BxError(s2, bx.lib().bx_last_error().decode())
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ws * B * e2e_steps / e2e_s, "unit": "evals/s", "h2d_bytes_per_step": B * P * 8,
           "d2h_bytes_per_step": B * 8 + B * P * 8}

    # the FP64 GPU form of the same evaluation
    B64 = min(B, 256)
    m64 = bx.Model(spec, precision=bx.BX_FP64, max_batch=B64, stream=stream)
    th64 = theta[:B64].contiguous()
    m64.nll_batch(th64, grad=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        m64.nll_batch(th64, grad=True)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_value = ws * B64 * 3 / (e0.elapsed_time(e1) / 1e3)
    m64.close()

    # the tensor-core species-resolved form (BX_TF32X3) of the same evaluation
    mtc = bx.Model(spec, precision=bx.BX_TF32X3, max_batch=B, stream=stream)
    mtc.nll_batch(theta, grad=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        mtc.nll_batch(theta, grad=True)
    e1.record(stream)
    torch.cuda.synchronize()
    tc_value = ws * B * 5 / (e0.elapsed_time(e1) / 1e3)
    mtc.close()
    return e2e, fp64_value, tc_value


def toy_fits(bx, I, n_toys, stream):
    """Batched pseudo-experiments: n_toys ragged toys (bins U{400..1200} of 2 npe from 150 npe,
    6-15 of the 15 library shapes, 1e4-1e7 events, Poisson data at theta_true), every toy
    fitted from theta_true (1 + 0.05 z) in one bx_fit call (FP32, one CUDA graph replayed
    until every fit has finished).  Wall time of the call (host clock, warm model)."""
    base = I.toy_batch(n_toys=n_toys, seed=7)
    gen = bx.Model([b.with_counts(np.zeros(b.n_bins_total)) for b in base], precision=bx.BX_FP32)
    specs = [b.with_counts(I.poisson_counts(gen.expected(b.theta_true, t), 1000 + t)) for t, b in enumerate(base)]
    gen.close()
    P = 7 + max(t.K for t in specs)
    th0 = np.zeros((n_toys, P))
    for t, sp in enumerate(specs):
        th0[t, : sp.P] = I.parameter_points(sp.theta_true, 1, rel=0.05, seed=300 + t, free=sp.default_free())[0]
    m = bx.Model(specs, precision=bx.BX_FP32, max_batch=n_toys * (8 + 2 * P), stream=stream)
    warm = min(n_toys, 64)
    m.fit(th0[:warm], toy_idx=np.arange(warm))   # workspace set-up (the graph is re-captured for n)
    t0 = time.perf_counter()
    out, info, st = m.fit(th0, toy_idx=np.arange(n_toys))
    wall = time.perf_counter() - t0
    m.close()
    ok = sum(1 for r in info if r["status"] == bx.BX_OK)
    evals = sum(r["n_evals"] for r in info)
    return {"toys": n_toys, "wall_s": wall, "fits_per_s": n_toys / wall, "converged": ok,
            "evals": int(evals), "evals_per_s": evals / wall, "precision": "BX_FP32",
            "recipe": "bins U{400..1200} x 2 npe from 150 npe, 6-15 species, 1e4-1e7 events, start theta_true (1 + 0.05 z)"}


DISCRIMINATION = ("discrimination: K=15, TFC 2x900 + energy x radius 900x60 + energy x pulse-shape 900x50 "
                  "(100800 bins), 22 parameters, 2e6 events")
JOINT = ("energy x radius x pulse-shape: K=15, TFC 2x900 + the 900 x 12 x 10 joint histogram of the vetoed "
         "events (109800 bins), 22 parameters, 2e6 events")


def discrimination_leg(bx, I, stream, B=256, steps=5, name="discrimination", workload=DISCRIMINATION, n_slices=112):
    """A 2D-slice model on the tensor cores: the discrimination regime (K = 15; TFC spectra and
    the 900 x 60 energy x radius and 900 x 50 energy x pulse-shape histograms, 100800 bins, 22
    parameters) or the joint energy x radius x pulse-shape grid (12 x 10 cells): -lnL + gradient
    evaluations/s (FP32 model, TF32 split GEMMs), the forward GEMM's tensor throughput, and the
    wall time of one fit."""
    import torch
    s = I.config(name)
    gen = bx.Model(s.with_counts(np.zeros(s.n_bins_total)), precision=bx.BX_FP32, stream=stream)
    s = s.with_counts(I.poisson_counts(gen.expected(s.theta_true), 0))
    gen.close()
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=B, stream=stream)
    pts = I.parameter_points(s.theta_true, B, rel=0.02, seed=400, free=s.default_free())
    dev = torch.device("cuda", torch.cuda.current_device())
    theta = torch.tensor(pts, dtype=torch.float64, device=dev)
    nll = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty((B, m.P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        st = bx.lib().bx_nll_batch(m.h, B, None, bx._ptr(theta), bx._ptr(nll), bx._ptr(grad), 1)
        if st:
            raise bx.BxError(st, bx.lib().bx_last_error().decode())

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    m.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    stage_ms, n_evals, entries = m.profile(False)
    per = {k: v / max(n_evals, 1) for k, v in stage_ms.items()}
    # forward GEMM: algorithmic 2 * (in-band response entries) * slices per evaluation
    alg = 2.0 * entries / max(n_evals, 1) * n_slices
    peaks = measured_peaks()
    tf32_peak = peaks.get("bf16_tflops", 1887.0) * (1.1 / 2.25)
    tc = alg / (per["forward"] / 1e3) / 1e12
    # one fit of the full model
    mf = bx.Model(s, precision=bx.BX_FP32, max_batch=8 + 2 * s.P, stream=stream)
    th0 = I.parameter_points(s.theta_true, 1, rel=0.1, seed=401, free=s.default_free())
    mf.fit(th0)
    t0 = time.perf_counter()
    _, info, st = mf.fit(th0)
    fit_s = time.perf_counter() - t0
    mf.close()
    m.close()
    return {"workload": workload, "global_batch": B,
            "value": B * steps / (total / 1e3), "unit": "evals/s", "ms_per_step": total / steps,
            "stage_ms_per_launch": {k: round(v, 4) for k, v in per.items()},
            "forward_gemm": {"bound": "tensor", "achieved": tc, "peak": tf32_peak, "unit": "TFLOP/s",
                             "frac": tc / tf32_peak,
                             "peak_basis": "measured bf16 burst x nominal TF32/BF16 ratio 1.1/2.25",
                             "algorithmic": f"2 x in-band response entries x {n_slices} slices per evaluation, over the "
                                            "forward stage (templates + generation + GEMM)"},
            "fit": {"wall_s": fit_s, "status": int(st), "evals": int(info[0]["n_evals"])}}


QUENCHED = ("multivariate with species-specific quenching (alpha at 2.3 MeV, 150 kB): 2 quenching "
            "groups of 2000 response columns")
SLICED = ("multivariate with the radial and pulse-shape terms in 3 energy slices (100-250, 250-500, "
          "500-1000 npe): 3 x (60 radial + 50 pulse-shape) bins")


def variant_leg(bx, I, name, workload, stream, B=2736, steps=5):
    """A variant of the multivariate model (species-specific quenching: the alpha species at
    2.3 MeV true energy quenched with 150 kB, with its own Birks map and response columns; or
    the Eq. 4 terms in several energy slices): -lnL + gradient evaluations/s at the main leg's
    batch, FP32, and one FP32 fit."""
    import torch
    s = make_dataset(bx, I, I.config(name), seed=0)
    m = bx.Model(s, precision=bx.BX_FP32, max_batch=B, stream=stream)
    pts = I.parameter_points(s.theta_true, B, rel=0.02, seed=410, free=s.default_free())
    dev = torch.device("cuda", torch.cuda.current_device())
    theta = torch.tensor(pts, dtype=torch.float64, device=dev)
    nll = torch.empty(B, dtype=torch.float64, device=dev)
    grad = torch.empty((B, m.P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        st = bx.lib().bx_nll_batch(m.h, B, None, bx._ptr(theta), bx._ptr(nll), bx._ptr(grad), 1)
        if st:
            raise bx.BxError(st, bx.lib().bx_last_error().decode())

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    m.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        total += e0.elapsed_time(e1)
    stage_ms, n_evals, _ = m.profile(False)
    per = {k: v / max(n_evals, 1) for k, v in stage_ms.items()}
    m.close()
    mf = bx.Model(s, precision=bx.BX_FP32, max_batch=8 + 2 * s.P, stream=stream)
    th0 = I.parameter_points(s.theta_true, 1, rel=0.05, seed=411, free=s.default_free())
    mf.fit(th0)
    t0 = time.perf_counter()
    _, info, st = mf.fit(th0)
    fit_s = time.perf_counter() - t0
    mf.close()
    return {"workload": workload, "global_batch": B,
            "value": B * steps / (total / 1e3), "unit": "evals/s", "ms_per_step": total / steps,
            "stage_ms_per_launch": {k: round(v, 4) for k, v in per.items()},
            "fit": {"wall_s": fit_s, "status": int(st), "evals": int(info[0]["n_evals"])}}


def fit_times(bx, I, spec, stream):
    """Full-fit wall time of one multivariate fit started at theta_true (1 + 0.1 z): FP32, FP64,
    and FP32 polished by FP64 (host wall clock around bx_fit, second call on a warm model)."""
    th0 = I.parameter_points(spec.theta_true, 1, rel=0.1, seed=200, free=spec.default_free())
    out = {"start": "theta_true * (1 + 0.1 z), 21 free parameters", "timing": "warm model, host wall clock"}
    models = {}
    for name, prec in (("fp32", bx.BX_FP32), ("fp64", bx.BX_FP64)):
        m = bx.Model(spec, precision=prec, max_batch=8 + 2 * spec.P, stream=stream)
        m.fit(th0)   # first call: workspace and graph set-up
        t0 = time.perf_counter()
        th, info, st = m.fit(th0)
        out[name + "_s"] = time.perf_counter() - t0
        out[name + "_status"] = int(st)
        out[name + "_evals"] = int(info[0]["n_evals"])
        out[name + "_nll"] = float(info[0]["nll"])
        models[name] = (m, th)
    m64, _ = models["fp64"]
    th32 = models["fp32"][1]
    t0 = time.perf_counter()
    th, info, st = m64.fit(th32)
    out["mixed_s"] = out["fp32_s"] + (time.perf_counter() - t0)
    out["mixed_status"] = int(st)
    out["mixed_nll"] = float(info[0]["nll"])
    out["d2nll_fp32_vs_fp64"] = 2.0 * abs(out["fp32_nll"] - out["fp64_nll"])
    for m, _ in models.values():
        m.close()
    return out


def report(args, ws, B, total_ms, value, stage_ms, n_evals, entries, e2e, fp64_value, tc_value, clk, fits=None,
           disc=None):
    # roofline of the dominant kernel (ALU-bound: FP32 issue rate of 152 SMs x 128 lanes)
    per_launch = {k: v / max(n_evals, 1) for k, v in stage_ms.items()}
    dom = max(("forward", "adjoint"), key=lambda k: per_launch[k])
    ops = (FWD_OPS_PER_ENTRY if dom == "forward" else BWD_OPS_PER_ENTRY) * entries / max(n_evals, 1)
    peak = SMS * FP32_LANES * SM_MAX_MHZ * 1e6 / 1e12
    achieved = ops / (per_launch[dom] / 1e3) / 1e12
    roofline = {"bound": "alu", "kernel": "k_fwd_f32" if dom == "forward" else "k_bwd_f32",
                "achieved": achieved, "peak": peak, "unit": "Top/s", "frac": achieved / peak,
                "traffic": TRAFFIC_PER_ITEM["k_fwd_f32" if dom == "forward" else "k_bwd_f32"] * B,
                "entries_per_launch": entries / max(n_evals, 1),
                "ops_per_entry": FWD_OPS_PER_ENTRY if dom == "forward" else BWD_OPS_PER_ENTRY,
                "peak_basis": "FP32 issue rate 152 SMs x 128 lanes x 2070 MHz (derived, not measured)",
                "stage_ms_per_launch": {k: round(v, 4) for k, v in per_launch.items()}}
    cb = None if args.no_cpu_baseline else cpu_baseline("multivariate", args.cpu_seconds)
    line = {"metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": ws * B, "precision": "BX_FP32 (FP64 columns, -lnL)",
                       "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "fp64_gpu_value": fp64_value, "mixed_over_fp64": value / fp64_value if fp64_value else None,
            "tf32x3_gpu_value": tc_value,
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "fit": fits, "discrimination_2d": disc,
            "gpu_launches": 5 * args.steps, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    # 2736 = 152 SMs x 18: whole waves for the forward (8 tiles per item at 18 CTAs per SM), the
    # column stage (one CTA per item at 3 per SM) and the assembly (one per item at 2 per SM)
    ap.add_argument("--batch", type=int, default=2736)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e, FP64 and fit legs (profiling runs)")
    ap.add_argument("--toys", type=int, default=4096, help="batched toy fits in the fit leg (0: none)")
    ap.add_argument("--batch2d", type=int, default=256, help="batch of the 2D-model leg (0: none)")
    ap.add_argument("--quenched", type=int, default=1, help="species-quenching leg (0: none)")
    ap.add_argument("--sliced", type=int, default=1, help="energy-sliced Eq. 4 leg (0: none)")
    ap.add_argument("--joint", type=int, default=1, help="energy x radius x pulse-shape leg (0: none)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
