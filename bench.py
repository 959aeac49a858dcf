#!/usr/bin/env python
"""Benchmark of the SMC-NUTS hot path: grad-lnL evaluations per second and
SMC-NUTS run time, mixed precision vs FP64, on the 11-D aligned-spin TaylorF2
workload (3 detectors, 8 s at 1/8 Hz, 8033 bins, 2048 particles, NUTS depth 6).

One step = one full SMC run (prior draw, then stages of adaptive reweighting,
ESS root-find, evidence increment, covariance, systematic resampling and
gather, and 2 NUTS transitions per particle until beta = 1), i.e. every step
of the hot path over one synthetic event. value = gradient evaluations (one
leapfrog of one particle = one ln L + gradient over all detectors and active
bins) per second, summed over ranks (one independent event per GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl sharpy|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grad-lnL evals/s and SMC-NUTS run time, mixed vs FP64 on GB300, |ΔlnZ|≤2σ"
UNIT = "evals/s"
# Algorithmic work per active (bin, detector) of the gradient sweep with 3
# detectors (FMA = 2 FLOP). Carrier and moments (all paths): angle scale 1,
# complex multiply 6, moments 9 x 4 + 2 -> 45 FLOP (FP32 in the mixed paths).
# mixed: the four large post-Newtonian terms as 4 FP64 FMA per bin shared by
#        3 detectors, the four small ones as FP32 split products (~13.5 FLOP
#        each) per bin, the delay term in FP32 per detector.
# split: FP32 phase, 8 split products per bin shared by 3 detectors + ~15
#        FLOP per detector -> 51 FLOP, total 96 FP32 FLOP.
# fp64: all eight terms in FP64 FMA, carrier by sincospi (~30 FMA), moments in FP64.
# These estimates stand in only while no instruction counts of the current
# kernel sources are recorded (COUNTED below).
def work(precision, n_det=3):
    """Estimated FLOP per active (bin, detector) of the gradient sweep with n_det detectors."""
    poly64 = 2.0 * 8.0 / n_det                   # FP64 FMA: the 8-term PN polynomial, once per bin for all detectors
    delay32 = 15.0                               # FP32: f tau_a from hi/lo splits, per detector
    phase32 = 8.0 * 13.5 / n_det + delay32       # split FP32 phase: 8 split products per bin + the delay term
    if precision == "mixed":
        return {"pipe": "fp64", "flop": 2.0 * 4.0 / n_det, "fp32_flop": 4.0 * 13.5 / n_det + delay32 + 45.0}
    if precision == "split":
        return {"pipe": "fp32", "flop": phase32 + 45.0, "fp32_flop": phase32 + 45.0}
    return {"pipe": "fp64", "flop": poly64 + 2.0 + 60.0 + 45.0, "fp32_flop": 0.0}


WORK = {p: work(p) for p in ("mixed", "split", "fp64")}


# Counter-derived work and traffic, valid only for the kernel sources they
# were taken on (reported while the sources' hash matches, else the estimates
# above and traffic null). From one ncu launch each (`--mode nuts_launch
# --ensemble late` for the NUTS kernel on the 11-D workload, `--mode
# loglike_launch` with the tuned `--split` for the likelihood kernels):
# FP64 FLOP = 2 DFMA + DADD + DMUL and FP32 FLOP = 2 FFMA + FADD + FMUL thread
# instructions (smsp__sass_thread_inst_executed_op_*_pred_on.sum) per active
# (bin, detector), and DRAM bytes read + written per launch.
# Each kernel's counts are keyed to the device-code files its instructions
# come from (context.cuh, the host-side context, is not among them).
COUNTED_SOURCES = {"nuts": ["nuts_kernel.cuh", "sweep.cuh", "physics.cuh", "common.cuh", "dfloat.cuh"],
                   "loglike": ["loglike_kernel.cuh", "split_stage.cuh", "bulk.cuh", "sweep.cuh", "physics.cuh",
                               "common.cuh", "dfloat.cuh"]}
COUNTED = {"sources_sha256_16": {"nuts": "4c9bc0a722a82040", "loglike": "43066a7c70b78fc5"},
           "nuts": {"mixed": {"fp64": 2.9620, "fp32": 107.01},
                    "split": {"fp64": 0.2756, "fp32": 126.67},
                    "fp64": {"fp64": 110.50, "fp32": 0.0152}},
           # the likelihood kernels, one call each with the tuner's choice for
           # that shape: 2048 vectors of the 11-D workload (1 warp per vector),
           # 8192 vectors of the 259585-bin segment (mixed and split: the staged
           # kernel; FP64: 4 warps per vector)
           "loglike": {"bbh11": {"mixed": {"fp64": 2.8057, "fp32": 88.321}},
                       "bns": {"mixed": {"fp64": 2.6686, "fp32": 81.405},
                               "split": {"fp64": 0.0019, "fp32": 101.07},
                               "fp64": {"fp64": 90.365, "fp32": 0.0}}},
           "traffic": {"mixed": 3830016, "split": 3913984, "fp64": 4599040},
           # the same captures: FP64 pipe busy, warps active and issue active
           # (sm__inst_executed_pipe_fp64, sm__warps_active,
           # smsp__issue_active; % of peak sustained active)
           "util": {"mixed": {"fp64_pipe": 34.4, "warps_active": 10.7, "issue_active": 37.0},
                    "split": {"fp64_pipe": 16.6, "warps_active": 10.7, "issue_active": 40.2},
                    "fp64": {"fp64_pipe": 86.0, "warps_active": 11.0, "issue_active": 8.0}}}


def _sources_hash(kernel="nuts"):
    import hashlib
    h = hashlib.sha256()
    for f in COUNTED_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2601_02336_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def counted(kernel, precision, workload="bbh11"):
    """(fp64 FLOP, fp32 FLOP, source) per active (bin, detector) of `kernel` ('nuts', or 'loglike' on `workload`)."""
    table = COUNTED[kernel] if kernel == "nuts" else COUNTED[kernel].get(workload, {})
    same = COUNTED["sources_sha256_16"][kernel] == _sources_hash(kernel)
    if same and precision in table:
        c = table[precision]
        return c["fp64"], c["fp32"], "ncu instruction counts of this kernel's sources"
    wk = WORK[precision]
    f64 = wk["flop"] if wk["pipe"] == "fp64" else 0.0
    why = "no counts recorded" if same else "sources changed since the counts"
    return f64, wk["fp32_flop"] if wk["pipe"] == "fp64" else wk["flop"], f"hand estimate ({why})"


def _traffic(precision):
    if COUNTED["sources_sha256_16"]["nuts"] != _sources_hash("nuts"):
        return None
    return COUNTED["traffic"].get(precision)


def _util(precision):
    if COUNTED["sources_sha256_16"]["nuts"] != _sources_hash("nuts"):
        return None
    return COUNTED["util"].get(precision)


def binding_pipe(f64, f32, p64, p32):
    """(pipe, FLOP per unit, peak) of the pipe that bounds a kernel doing f64 FP64 and f32 FP32 FLOP per unit:
    the one whose work takes longer at its peak (the two pipes issue concurrently)."""
    if p32 and f32 / p32 > f64 / p64:
        return "fp32", f32, p32
    return "fp64", f64, p64


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.first = 0

    def start(self):
        """Start sampling every 50 ms; returns once the first sample is in (at most 3 s), so that the timed
        region that follows is sampled from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
            return
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self):
        """The timed region starts: later samples are the ones reported (earlier ones only if none came)."""
        self.first = len(self.lines)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.first:] or self.lines[-1:]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(name):
    from paper_2601_02336_gb300 import inputs
    return inputs.WORKLOADS[name]()


def _describe(w):
    metric = {0: "identity metric", 1: "covariance metric", 2: "per-particle local metric"}[w.metric]
    det = "1 detector (F+ = 1)" if w.fixed_response else f"{w.n_det} detectors"
    return (f"{w.name}: {w.n_dim}-D TaylorF2, {det}, {1.0 / w.df:g} s at 1/{1.0 / w.df:g} Hz "
            f"({w.n_bins} bins, {w.f_min:g}-{w.f_max:g} Hz), {w.n_particles} particles, NUTS depth {w.max_depth}, "
            f"alpha {w.alpha}, {w.n_mut} transitions/stage, {metric}; one step = one full SMC run")


def _oracle_sample(n_particles, seed, name="bbh11", max_depth=None):
    """A bounded sample of the workload for the oracle: one NUTS transition of
    n_particles particles of the same event at beta = 0.5 (mid-run state)."""
    import oracle
    from paper_2601_02336_gb300 import inputs
    from tests import helpers
    w = _workload(name)
    ev, th_inj, _ = helpers.make_event(w, seed=0)
    model = helpers.oracle_model(w)
    th = inputs.ball(w, th_inj, n_particles, 500 + seed, rel=1e-3)
    lnl, g = oracle.loglike(model, ev, th)
    sig = np.std(th, axis=0)
    eps = 0.5 * float(np.min(sig))
    depth = w.max_depth if max_depth is None else max_depth
    t0 = time.perf_counter()
    _, _, _, st = oracle.nuts_mutate(model, ev, 0.5, th, lnl, g, None, eps, depth, 1, key=77 + seed, ctr=1)
    dt = time.perf_counter() - t0
    return int(st["n_leapfrog"].sum()), dt


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count()
    n_part = 8 * cores
    for i in range(args.warmup):
        _oracle_sample(n_part, i)
    evals, secs = 0, 0.0
    for k in range(args.steps):
        e, dt = _oracle_sample(n_part, 100 + k)
        evals += e
        secs += dt
    v = evals / secs
    sample = (f"oracle NUTS, one transition of {n_part} particles per step at beta=0.5 near the injection, "
              f"bbh11 event (8033 bins x 3 detectors), OpenMP over particles")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "bbh11 (bounded oracle sample)"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def _active_bins(w, th):
    """(bins with f_k <= f_ISCO) x detectors per parameter vector (reporting only)."""
    from paper_2601_02336_gb300 import inputs
    tsun = 4.925491025543576e-6
    ph = np.tile(np.array(w.fixed, dtype=np.float64), (th.shape[0], 1))
    ph[:, w.phys] = th
    mc, q = ph[:, inputs.MC], ph[:, inputs.Q]
    eta = q / (1.0 + q) ** 2
    m = mc * eta ** -0.6
    fisco = 1.0 / (6.0 ** 1.5 * math.pi * m * tsun)
    k = np.clip(np.floor((fisco - w.f_min) / w.df), -1, w.n_bins - 1)
    return (k + 1) * w.n_det


def main_loglike(args):
    """sharpy_loglike_grad throughput (one call = ln L + gradient of N particles)
    on two parameter sets of a workload: prior draws and a Gaussian ball around
    the injection (sigma = 1e-3 x prior width); FP64, mixed and split paths;
    the oracle's rate on 64 of the ball's vectors (1 thread and all threads) and
    the mixed path's largest |d lnL| against it. One JSON line per workload."""
    import torch

    import oracle
    from paper_2601_02336_gb300 import api, inputs
    from paper_2601_02336_gb300._lib import lib
    from tests import helpers

    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[args.workload]()
    ctx, th_inj, data = api.make_event(w, seed=0)
    n = max(w.n_particles, 2048)
    sets = {"prior": inputs.prior_draws(w, n, 1), "ball": inputs.ball(w, th_inj, n, 2, rel=1e-3)}
    peaks = (C.c_double * 3)()
    lib().sharpy_probe_peaks(0, peaks)
    stream = torch.cuda.current_stream()
    out = {"mode": "loglike", "workload": w.name, "n_bins": w.n_bins, "n_det": w.n_det, "particles_per_call": n,
           "fp32_peak_tflops": peaks[0], "fp64_peak_tflops": peaks[1], "sets": {}}
    for name, th in sets.items():
        t = torch.tensor(th, dtype=torch.float64, device="cuda")
        act = float(_active_bins(w, th).mean())
        row = {"active_bin_det_per_eval": act}
        for prec in ("fp64", "mixed", "split"):
            for _ in range(2):
                ctx.loglike_grad(t, prec)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                ctx.loglike_grad(t, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            f64c, f32c, fsrc = counted("loglike", prec, w.name)
            pipe, flop, peak = binding_pipe(f64c, f32c, peaks[1], peaks[0])
            tfl = n * act * flop / (ms * 1e-3) / 1e12
            row[prec] = {"evals_per_s": n / (ms * 1e-3), "ms_per_call": ms, "pipe": pipe,
                         "flop_per_active_bin_det": flop, "flop_source": fsrc,
                         "achieved_tflops": tfl, "frac": tfl / peak,
                         "warps_per_vector_tuned": ctx.loglike_split(n, prec)}
        out["sets"][name] = row
    # oracle on 64 vectors of the ball set, and the mixed path's error against it
    oracle.build()
    model = helpers.oracle_model(w)
    ev, _, odata = helpers.make_event(w, seed=0)
    sub = sets["ball"][:64]
    cores = os.cpu_count()
    rates = {}
    for threads in (1, cores):
        prev = oracle.set_threads(threads)
        t0 = time.perf_counter()
        lref, gref = oracle.loglike(model, ev, sub)
        rates[threads] = len(sub) / (time.perf_counter() - t0)
        oracle.set_threads(prev)
    # the same arrays on both sides: the oracle's event staged into a second context
    ctx2 = api.Context.from_workload(w)
    ctx2.set_data(odata, inputs.psd_array(w), w.f_min, w.df, inputs.detectors(w))
    lm, gm = ctx2.loglike_grad(torch.tensor(sub, dtype=torch.float64, device="cuda"), "mixed")
    out["oracle"] = {"evals_per_s_1_thread": rates[1], "evals_per_s_all": rates[cores], "cores": cores,
                     "sample": "64 vectors of the ball set"}
    out["mixed_max_abs_dlnl_vs_oracle"] = float(np.max(np.abs(lm.cpu().numpy() - lref)))
    print(json.dumps(out))
    return 0


def _extra_workloads(args, flush):
    """The other single-GPU workloads, measured after the timed region (CUDA events, L2 flushed before each
    timed call): one bbh11_long SMC run per precision (16384 particles, covariance metric, after one untimed
    run that also tunes the slot count), sharpy_loglike_grad on 8192 near-injection vectors of the 259585-bin
    bns event (mixed and FP64), and one batched run of the 64-event batch64 workload (after one untimed run
    that tunes it)."""
    import torch

    from paper_2601_02336_gb300 import api, inputs
    stream = torch.cuda.current_stream()

    def timed(fn):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    out = {}
    w = inputs.bbh11_long()
    ctx, _, _ = api.make_event(w, seed=0)
    ra = (w.n_particles, w.alpha, w.n_mut, w.max_depth, w.metric, w.eps_scale)
    row = {"workload": _describe(w)}
    for prec in ("mixed", "fp64"):
        ctx.smc_run(*ra, key=40_000, precision=prec)
        (lnz, _, _, rec), ms = timed(lambda: ctx.smc_run(*ra, key=40_001, precision=prec))
        ev = sum(r["n_leapfrog"] for r in rec)
        row[prec] = {"ms_per_run": ms, "evals_per_s": ev / (ms * 1e-3), "stages": len(rec), "lnz": lnz}
    out["bbh11_long_smc_run"] = row
    del ctx
    w = inputs.bns()
    ctx, th_inj, _ = api.make_event(w, seed=0)
    th = torch.tensor(inputs.ball(w, th_inj, 8192, 2, rel=1e-3), dtype=torch.float64, device="cuda")
    row = {"workload": "bns: 259585 bins x 3 detectors, 8192 vectors near the injection (sigma 1e-3 of the "
                       "prior width), one sharpy_loglike_grad call = ln L + gradient of all 8192",
           "active_bin_det_per_eval": float(_active_bins(w, th.cpu().numpy()).mean())}
    for prec in ("mixed", "split", "fp64"):
        ctx.loglike_grad(th, prec)  # the first call of this shape tunes the warps per vector
        _, ms = timed(lambda: ctx.loglike_grad(th, prec))
        row[prec] = {"ms_per_call": ms, "evals_per_s": 8192 / (ms * 1e-3),
                     "warps_per_vector_tuned": ctx.loglike_split(8192, prec)}
    out["bns_loglike_grad"] = row
    del ctx, th
    ws = inputs.batch64()
    ctxs = [api.make_event(wi, seed=i)[0] for i, wi in enumerate(ws)]
    w0 = ws[0]
    b = api.Batch(ctxs, [wi.n_particles for wi in ws], w0.alpha, w0.n_mut, w0.max_depth, w0.metric, w0.eps_scale,
                  precision="mixed", max_stages=500)
    b.run([50_000 + e for e in range(len(ws))])
    (res, rounds), ms = timed(lambda: b.run([60_000 + e for e in range(len(ws))]))
    out["batch64_run"] = {"workload": "batch64: 64 events, segments 4/8/16/32 s, 512-8192 particles, depth 8, "
                                      "mixed precision, one batched run of all 64 events",
                          "ms_per_run": ms, "events_per_hour": len(ws) / (ms * 1e-3) * 3600.0,
                          "evals_per_s": sum(r["n_leapfrog"] for r in res) / (ms * 1e-3), "rounds": rounds,
                          "slots": b.slots}
    b.close()
    del ctxs, b
    # the timed workload's event, 8 independent runs (keys) through the batched driver: in a single run most
    # stages' NUTS launches last as long as their slowest particle's trees, while batched the runs' tails overlap
    w = inputs.bbh11()
    R = 8
    ctxs = [api.make_event(w, seed=0)[0] for _ in range(R)]
    b = api.Batch(ctxs, [w.n_particles] * R, w.alpha, w.n_mut, w.max_depth, w.metric, w.eps_scale,
                  precision="mixed", max_stages=500)
    b.run([70_000 + e for e in range(R)])
    (res, rounds), ms = timed(lambda: b.run([80_000 + e for e in range(R)]))
    lz = [r["lnz"] for r in res]
    out["bbh11_runs_batched"] = {"workload": f"{R} independent runs of the timed workload's event (same data, "
                                             "keys differ) in one batched driver, mixed precision",
                                 "ms_per_batch": ms, "ms_per_run_equivalent": ms / R,
                                 "evals_per_s": sum(r["n_leapfrog"] for r in res) / (ms * 1e-3),
                                 "rounds": rounds, "slots": b.slots, "lnz_mean": float(np.mean(lz)),
                                 "lnz_sd": float(np.std(lz, ddof=1))}
    b.close()
    return out


def main_nuts_launch(args):
    """One persistent NUTS launch on fixed ensembles of an event (by default bbh11: 2048 particles, depth 6,
    two transitions, identity metric, step 0.5 x the ensemble's smallest standard deviation): "first" = prior
    draws at beta = 1e-4 (the first stage's regime: most trees reach the depth limit), "late" = a Gaussian
    ball around the injection (sigma 1e-3 of the prior width) at beta = 1 (a posterior-like stage). The
    launches are deterministic, so versions of the kernel are compared on identical work; also the command
    the instruction-count and DRAM captures of the roofline are taken on (--ensemble picks one; --workload,
    --particles and --depth change the event, the ensemble size and the tree depth)."""
    import torch

    from paper_2601_02336_gb300 import api, inputs
    torch.cuda.set_device(0)
    if args.workload not in inputs.WORKLOADS:
        raise SystemExit("nuts_launch runs one event")
    w = inputs.WORKLOADS[args.workload]()
    n = args.particles or w.n_particles
    depth = args.depth or w.max_depth
    ctx, th_inj, _ = api.make_event(w, seed=0)
    sets = {"first": (inputs.prior_draws(w, n, 1), 1e-4),
            "late": (inputs.ball(w, th_inj, n, 2, rel=1e-3), 1.0)}
    names = [args.ensemble] if args.ensemble else list(sets)
    if args.slots:
        ctx.set_nuts_slots(args.slots)
    stream = torch.cuda.current_stream()
    out = {"mode": "nuts_launch", "workload": _describe(w), "precision": args.precision, "ensembles": {}}
    for name in names:
        th, beta = sets[name]
        eps = 0.5 * float(np.min(np.std(th, axis=0)))
        t0 = torch.tensor(th, dtype=torch.float64, device="cuda")
        l0, g0 = ctx.loglike_grad(t0, "fp64")
        times, st = [], None
        for k in range(args.warmup + args.steps):
            t, l, g = t0.clone(), l0.clone(), g0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s = ctx.nuts_mutate(beta, t, l, g, None, eps, depth, w.n_mut, key=77, ctr=256,
                                precision=args.precision)
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
                st = api.Context.stats_to_numpy(s)
        import hashlib
        digest = hashlib.sha256(b"".join(a.cpu().numpy().tobytes() for a in (t, l, g))).hexdigest()[:16]
        out["ensembles"][name] = {"beta": beta, "step": eps, "ms_median": float(np.median(times)),
                                  "state_sha256_16": digest,
                                  "ms_min": float(np.min(times)), "launches": len(times),
                                  "active_bin_det": float(st["active_bins"].sum()),
                                  "n_leapfrog": int(st["n_leapfrog"].sum()),
                                  "accept_mean": float(st["accept_sum"].mean() / w.n_mut)}
    out["status"] = ctx.status()
    print(json.dumps(out))
    return 0


def main_loglike_launch(args):
    """One sharpy_loglike_grad call (ln L + gradient) on N vectors near the injection of a workload (sigma 1e-3 of
    the prior width), after one untimed call: the command the standalone likelihood kernel's instruction-count
    capture is taken on (--workload, --precision, --particles)."""
    import torch

    from paper_2601_02336_gb300 import api, inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS[args.workload]()
    ctx, th_inj, _ = api.make_event(w, seed=0)
    n = args.particles or w.n_particles
    th = torch.tensor(inputs.ball(w, th_inj, n, 2, rel=1e-3), dtype=torch.float64, device="cuda")
    if args.split:
        ctx.set_loglike_split(args.split)  # no tuning launches: the first call is one launch
    ctx.loglike_grad(th, args.precision)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.loglike_grad(th, args.precision)
    e1.record(stream)
    torch.cuda.synchronize()
    act = float(_active_bins(w, th.cpu().numpy()).sum())
    print(json.dumps({"mode": "loglike_launch", "workload": w.name, "precision": args.precision, "particles": n,
                      "split": ctx.loglike_split(n, args.precision) if not args.split else args.split,
                      "ms": e0.elapsed_time(e1), "active_bin_det": act, "status": ctx.status()}))
    return 0


def main_batch(args):
    """64 uneven events (4/8/16/32 s segments, 512-8192 particles, NUTS depth 8)
    sampled together by the batched driver: one step = one batched run of all
    64 events from their prior draws to beta = 1."""
    import torch
    import torch.distributed as dist

    from paper_2601_02336_gb300 import api, inputs, multirank

    rank, world, local = multirank.env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ws = inputs.batch64()
    if args.metric is not None:
        for w in ws:
            w.metric = args.metric
    base = multirank.event_seed(rank) * 1000
    ctxs = [api.make_event(w, seed=base + i, device=local)[0] for i, w in enumerate(ws)]
    w0 = ws[0]
    b = api.Batch(ctxs, [w.n_particles for w in ws], w0.alpha, w0.n_mut, w0.max_depth, w0.metric, w0.eps_scale,
                  precision=args.precision, max_stages=500)
    if args.slots:
        b.slots = args.slots
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for i in range(args.warmup):
        b.run([multirank.run_key(10_000 + 100 * i, rank, e) for e in range(len(ws))])
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    clocks.mark()
    evals, bins, rounds, step_ms, lnzs, launches = 0.0, 0.0, [], [], [], 0
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, nr = b.run([multirank.run_key(20_000 + 100 * k, rank, e) for e in range(len(ws))])
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        evals += sum(r["n_leapfrog"] for r in res)
        bins += sum(r["active_bins"] for r in res)
        rounds.append(nr)
        launches += b.launches
        lnzs.append([r["lnz"] for r in res])
    barrier()
    clk = clocks.stop()
    t_rank = sum(step_ms)
    t_max = multirank.reduce_scalar(t_rank, "max", world, device="cuda")
    total = multirank.reduce_scalar(evals, "sum", world, device="cuda")
    n_ev = len(ws) * args.steps * world
    if rank == 0:
        f64c, f32c, _ = counted("nuts", args.precision)
        wk = {"flop": f32c if args.precision == "split" else f64c}  # the pipe that binds on the 11-D workload
        out = {"metric": METRIC, "value": total / (t_max * 1e-3), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": {"mixed": "f32+f64", "split": "f32 (f64 per particle)", "fp64": "f64"}[args.precision],
               "data": "synthetic",
               "config": {"workload": "batch64: 64 events of the 11-D TaylorF2 model, segments 4/8/16/32 s "
                                      "(16 each, 20-1024 Hz at 1/T), 512-8192 particles (log-uniform), NUTS depth 8; "
                                      "one step = one batched run of all 64 events",
                          "precision": args.precision, "l2": "flushed (256 MB write) between steps",
                          "particles": int(sum(w.n_particles for w in ws)), "slots": b.slots,
                          "rounds_per_run": rounds},
               "events_per_hour": n_ev / (t_max * 1e-3) * 3600.0,
               "round_ms": t_max / max(sum(rounds), 1),
               "achieved_tflops_whole_step": bins * wk["flop"] / (t_rank * 1e-3) / 1e12,
               "gpu_launches": launches, "clocks": clk,
               "lnz_first_events": [float(x) for x in lnzs[0][:4]]}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sharpy", choices=["sharpy", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "split", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=16,
                    help="FP64 runs for the mixed-vs-FP64 comparison (ln Z within 2 combined standard errors)")
    ap.add_argument("--lnz-runs", type=int, default=16,
                    help="mixed runs for that comparison: the timed runs plus untimed ones up to this count")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the extra keys: the other single-GPU workloads, measured after the timed region")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="bbh11", choices=["tiny", "bbh11", "bbh11_long", "bns", "batch64"])
    ap.add_argument("--mode", default="smc", choices=["smc", "loglike", "nuts_launch", "loglike_launch"])
    ap.add_argument("--particles", type=int, default=0,
                    help="loglike_launch and nuts_launch: vectors per call (0: the workload's)")
    ap.add_argument("--depth", type=int, default=0, help="nuts_launch: NUTS tree depth (0: the workload's)")
    ap.add_argument("--split", type=int, default=0, choices=[0, 1, 2, 4, 8, 16],
                    help="loglike_launch: warps per vector, 16 = the staged kernel (0: tuned)")
    ap.add_argument("--ensemble", default=None, choices=["first", "late"], help="nuts_launch: one ensemble only")
    ap.add_argument("--slots", type=int, default=0, choices=[0, 4, 8, 16, 32],
                    help="NUTS particles per CTA (0: autotuned / default)")
    ap.add_argument("--metric", type=int, default=None, choices=[0, 1, 2],
                    help="NUTS metric (default: the workload's): 0 identity, 1 covariance, 2 per-particle local")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "loglike":
        return main_loglike(args)
    if args.mode == "nuts_launch":
        return main_nuts_launch(args)
    if args.mode == "loglike_launch":
        return main_loglike_launch(args)
    if args.workload == "batch64":
        return main_batch(args)

    import torch
    import torch.distributed as dist

    from paper_2601_02336_gb300 import api, inputs, multirank
    from paper_2601_02336_gb300._lib import lib

    rank, world, local = multirank.env_rank()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def allmax(x):
        return multirank.reduce_scalar(x, "max", world, device="cuda")

    def allsum(x):
        return multirank.reduce_scalar(x, "sum", world, device="cuda")

    w = inputs.WORKLOADS[args.workload]()
    if args.metric is not None:
        w.metric = args.metric
    ctx, th_inj, data = api.make_event(w, seed=multirank.event_seed(rank), device=local)
    if args.slots:
        ctx.set_nuts_slots(args.slots)
    run_args = (w.n_particles, w.alpha, w.n_mut, w.max_depth, w.metric, w.eps_scale)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2

    def one_run(key, precision, timing=True):
        return ctx.smc_run(*run_args, key=key, precision=precision, timing=timing)

    for i in range(args.warmup):
        one_run(multirank.run_key(10_000, rank, i), args.precision)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    clocks.mark()
    evals = 0
    bins = 0.0
    nuts_ms = 0.0
    rew_ms = 0.0
    launches = 0
    step_ms = []
    lnzs = []
    n_stages = []
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lnz, th, ll, rec = one_run(multirank.run_key(20_000, rank, k), args.precision)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        evals += sum(r["n_leapfrog"] for r in rec)
        bins += sum(r["active_bins"] for r in rec)
        nuts_ms += sum(r["nuts_ms"] for r in rec)
        rew_ms += sum(r["reweight_ms"] for r in rec)
        # prior draw and ln L, then per stage: reweight, covariance, systematic, save, gather, the
        # local metric (metric 2), NUTS, record (the slot tuner ran in the warm-up runs)
        launches += 2 + (7 + (1 if w.metric == 2 else 0)) * len(rec)
        lnzs.append(lnz)
        n_stages.append(len(rec))
    barrier()
    clk = clocks.stop()
    t_rank = sum(step_ms)
    t_max = allmax(t_rank)
    total_evals = allsum(evals)
    value = total_evals / (t_max * 1e-3)

    # roofline of the dominant kernel (persistent NUTS), from its in-run durations
    peaks = (C.c_double * 3)()
    lib().sharpy_probe_peaks(local, peaks)
    fp32_peak, fp64_peak = peaks[0], peaks[1]
    f64c, f32c, fsrc = counted("nuts", args.precision)
    pipe, flop, peak = binding_pipe(f64c, f32c, fp64_peak, fp32_peak)
    secs = nuts_ms * 1e-3
    ach = bins * flop / secs / 1e12
    fp64_ach, fp32_ach = bins * f64c / secs / 1e12, bins * f32c / secs / 1e12
    kname = {"mixed": "MIXED", "split": "MIXED_SPLIT", "fp64": "FP64"}[args.precision]
    roofline = {"bound": "alu", "kernel": f"nuts_kernel<{kname},{w.n_det}>", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak if peak else None,
                "traffic": _traffic(args.precision) if w.name == "bbh11" else None,
                "traffic_unit": "bytes per NUTS launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "pipe": pipe, "flop_per_active_bin_det": flop, "flop_source": fsrc,
                "fp64_flop_per_active_bin_det": f64c, "fp32_flop_per_active_bin_det": f32c,
                "peak_source": f"measured {pipe.upper()} FMA probe on this GPU (sharpy_probe_peaks)",
                "fp64_achieved": fp64_ach, "fp64_frac": fp64_ach / fp64_peak if fp64_peak else None,
                "fp32_achieved": fp32_ach, "fp32_peak": fp32_peak,
                "fp32_frac": fp32_ach / fp32_peak if fp32_peak else None, "fp64_peak": fp64_peak,
                "ncu_pipe_utilisation_pct": _util(args.precision) if w.name == "bbh11" else None,
                "nuts_share_of_step": nuts_ms / t_rank,
                "reweight_share_of_step": rew_ms / t_rank,
                "active_bin_det_per_eval": bins / max(evals, 1)}

    # the other precision for the mixed-vs-FP64 comparison and |d lnZ| <= 2 sigma
    other = {}
    if args.fp64_steps > 0 and args.precision != "fp64":
        ev_o, t_o, lz_o = 0, 0.0, []
        for k in range(args.fp64_steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lnz, th, ll, rec = one_run(multirank.run_key(30_000, rank, k), "fp64")
            e1.record(stream)
            torch.cuda.synchronize()
            t_o += e0.elapsed_time(e1)
            ev_o += sum(r["n_leapfrog"] for r in rec)
            lz_o.append(lnz)
        # the timed runs' ln Z plus untimed runs of the same precision (keys continuing), so that each side of
        # the 2-sigma comparison has at least --lnz-runs runs
        lz_m = [float(x) for x in lnzs]
        for k in range(args.steps, args.lnz_runs):
            lz_m.append(one_run(multirank.run_key(20_000, rank, k), args.precision, timing=False)[0])
        se_m = np.std(lz_m, ddof=1) / math.sqrt(len(lz_m)) if len(lz_m) > 1 else float("nan")
        se_f = np.std(lz_o, ddof=1) / math.sqrt(len(lz_o)) if len(lz_o) > 1 else float("nan")
        other = {"fp64_value": ev_o / (t_o * 1e-3), "fp64_ms_per_step": t_o / args.fp64_steps,
                 "speedup_mixed_over_fp64": value / world / (ev_o / (t_o * 1e-3)),
                 "lnz_mixed": lz_m, "lnz_fp64": [float(x) for x in lz_o],
                 "dlnz": float(np.mean(lz_m) - np.mean(lz_o)),
                 "two_sigma": float(2.0 * math.sqrt(se_m ** 2 + se_f ** 2))}
        gold = os.path.join(ROOT, "tests", "golden", f"lnz_{w.name}_oracle.json")
        gold_cfg = None
        if os.path.exists(gold):
            with open(gold) as fh:
                gold_cfg = json.load(fh)
        same_sampler = gold_cfg is not None and all(
            gold_cfg.get(k) == v for k, v in (("metric", w.metric), ("n_particles", w.n_particles),
                                              ("max_depth", w.max_depth), ("n_mut", w.n_mut), ("alpha", w.alpha),
                                              ("eps_scale", w.eps_scale)))
        if same_sampler and world == 1:
            # ln Z of the oracle's own full runs on this event with the same sampler settings (stored by
            # tests/golden/make_lnz_oracle.py; the same injection and noise, its waveform from the oracle instead
            # of the library: ~1e-12 apart)
            ref = [r["lnz"] for r in gold_cfg["runs"]]
            se_r = np.std(ref, ddof=1) / math.sqrt(len(ref))
            other["vs_oracle"] = {
                "oracle_runs": len(ref), "oracle_mean": float(np.mean(ref)),
                "dlnz_mixed": float(np.mean(lz_m) - np.mean(ref)),
                "two_sigma_mixed": float(2.0 * math.sqrt(se_m ** 2 + se_r ** 2)),
                "dlnz_fp64": float(np.mean(lz_o) - np.mean(ref)),
                "two_sigma_fp64": float(2.0 * math.sqrt(se_f ** 2 + se_r ** 2))}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        psd = inputs.psd_array(w)
        dets = inputs.detectors(w)
        h_data = torch.from_numpy(np.ascontiguousarray(data)).pin_memory()
        h_psd = torch.from_numpy(np.ascontiguousarray(psd)).pin_memory()
        e_evals, e_secs = 0, 0.0
        K = w.n_bins
        # a new event on the same grid: the pre-whitened data (FP64 and FP32) and the prefix table are copied
        h2d = w.n_det * K * (16 + 8 + 8)
        d2h = 0
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.set_data(h_data.numpy(), h_psd.numpy(), w.f_min, w.df, dets)
            # the keys of the device-timed runs: the same runs, so the two numbers differ by the API's overhead
            lnz, th, ll, rec = one_run(multirank.run_key(20_000, rank, k), args.precision, timing=False)
            th_h = th.cpu()
            ll_h = ll.cpu()
            torch.cuda.synchronize()
            e_secs += time.perf_counter() - t0
            e_evals += sum(r["n_leapfrog"] for r in rec)
            d2h = th_h.numel() * 8 + ll_h.numel() * 8 + 8 * (9 * len(rec) + 2)
        e_max = allmax(e_secs)
        e2e = {"value": allsum(e_evals) / e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    extra = None
    if rank == 0 and world == 1 and not args.no_extra and args.workload == "bbh11":
        extra = _extra_workloads(args, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cores = os.cpu_count()
        # about 10-30 s of oracle work: fewer particles and a shallower tree on the long segments
        big = w.n_bins * w.n_det > 200_000
        n_part = cores if big else 8 * cores
        depth = 3 if big else w.max_depth
        e, dt = _oracle_sample(n_part, 0, w.name, depth)
        cpu = {"value": e / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"oracle NUTS, one transition (depth {depth}) of {n_part} particles at beta=0.5 near the "
                         f"injection of the same workload ({e} gradient evaluations, {dt:.1f} s)"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": {"mixed": "f32+f64", "split": "f32 (f64 per particle)", "fp64": "f64"}[args.precision],
               "data": "synthetic",
               "config": {"workload": _describe(w),
                          "precision": args.precision, "l2": "flushed (256 MB write) between steps",
                          "parallelism": f"one independent event per GPU x {world}",
                          "stages_per_run": n_stages},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clk, "mixed_vs_fp64": other,
               "lnz": {"mean": float(np.mean(lnzs)), "runs": [float(x) for x in lnzs]},
               "other_workloads": extra}
        print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
