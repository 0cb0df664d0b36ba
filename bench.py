#!/usr/bin/env python
"""Benchmark: cell-updates/s per artificial-compressibility time step.

Workload (headline): one Yin-Yang shell, 128x128x384 MAC cells per patch,
R1=0.5, R2=1, Pr=1, Ra=1e3, dt=5e-4, 3 Schwarz / splitting-error-reduction
iterations per step, FP64, forced by the trigonometric manufactured solution
with homogeneous walls (synthetic data, seeded, no dataset).  A cell-update is
one MAC cell of one patch advanced through one full AC step, all Schwarz
iterations included: value = 2 Nr Nth Nph * steps / time.

Timing: W untimed warm-up steps, then exactly K steps bracketed by
barrier + synchronize, timed with CUDA events on the solver's stream; the
state (~10 GB) is larger than L2, so no flush is needed.  N > 1: one
independent shell per GPU (replicas; no collective on the data path), value =
total cell-updates / max over ranks.

Also reported: e2e (the same metric through the C ABI with pinned host
buffers: upload both time levels, one step, download level 0, per step),
per-kernel times from CUDA events, roofline of the dominant kernel class,
SM clocks sampled during the timed region, and the FP64 oracle timed on the
host cores on a bounded sample (cpu_baseline).

By default (one GPU) the same JSON line also carries, as objects:
  mixed     the same shell in the mixed FP32/FP64 form (device and e2e
            rates, roofline, the line solves' fraction of HBM bandwidth);
  ensemble  64 seeded uneven shells in one batch (one launch per kernel
            class, a CUDA graph per step), 100 timed steps, per-class
            roofline, against the plain FP64 path one shell at a time;
  serving   200 Poisson-arriving requests (Nr <= 128, Nth <= 192,
            N in [50, 500] steps) under continuous batching at 0.8 of the
            batched capacity: p50/p99 time to completion, aggregate
            cell-updates/s, against FIFO plain FP64 service.
--workload shell|ensemble|serving runs one of them alone.

--impl reference runs the oracle (a plain CPU program; there is no other
implementation of the paper's method) on a bounded sample of the same
workload and prints the same line with "impl": "reference".
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per AC step"
UNIT = "cell-updates/s"

# Algorithmic traffic per cell per launch of each kernel class: (words of the
# storage type, FP64 words), one read of every input array and one write of
# every output (neighbour reuse on chip; ghosts ~1/N ignored).
#   extrapolate (per step): levels n, n-1 in (7 + 7 bulk, 2 + 2 pressures),
#     iterate out (7 + 2) and the advecting velocity out (3); then the sums
#     of the advecting velocity around each location: a in (3), 9 sums out
#   resid_T: T at both levels, 3 sums of the advecting velocity, forcing in,
#     B out
#   resid_u (average of 6): its system's 3 components at both levels, the
#     own advecting component and 2 sums of the others, forcing, B out, T at
#     both levels for u_r; the pressures entering the row: p1^n for system 1,
#     p2^n, p1, p1^n for 2
#   line solves (sweep_*): rhs, the three stored factors, result = 5; a final
#     factor also reads and writes the iterate = 6; averaged over the launches
#     of one iteration (r: 2 of 7 final, theta: 2 of 7, phi: 3 of 7)
#   pressure: 6 velocity values in; FP64: p^n, old and new p (system 1),
#     p2^n, p1, p1^n, old and new p2 (system 2)
#   factorize: advecting component in, three factors out
WORDS_PER_CELL = {
    "extrapolate": (36.0, 6.0), "resid_T": (7.0, 0.0), "resid_u": (35.0 / 3, 2.0), "sweep_r": (37.0 / 7, 0.0),
    "sweep_t": (37.0 / 7, 0.0), "sweep_p": (38.0 / 7, 0.0), "pressure": (6.0, 4.0), "factorize": (4.0, 0.0),
    # FP64 passes per iteration: T's sums (1 field), each velocity system's
    # three components (3 + 3 fields; read 2, write 1 word a field) and P2
    # (read 3, write 1 FP64 word): 4 launches
    "sums": (21.0 / 4, 4.0 / 4),
}
# FP64 operations per cell (hand count of the kernel formulas, FMA = 2, a
# division = 1) for the FP64 form, whose kernels are bound by the FP64 pipe.
# The sums of the advecting velocity are formed once per step (extrapolate
# class) and the two-level sums psi + psi^n of T and the velocity in their own
# class (sums), so neither is counted again in the residuals or the pressure.
FLOPS_PER_CELL = {"resid_T": 32.0, "resid_u": 68.0 - 2.0 / 3, "pressure": 15.0, "factorize": 9.0, "sums": 9.0 / 4}
FP64_PEAK_TFLOPS = 1.25   # nominal dense FP64 of GB300 (context; the bench measures its own)
# DRAM bytes (read + write) per point of the top kernel class from one ncu
# capture of its u_r launch on a smaller shell whose launch already exceeds L2
# (traffic scales with the points processed); the bench reports it scaled to
# one full launch.  Valid for the kernel code the capture was taken of.
TRAFFIC_PER_POINT = {
    (False, "resid_u"): (153.949e6 / (2 * 64 * 63 * 192), "profiles/k_resid_ur_fp64_64x64x192_full.md"),
    (True, "resid_u"): (518.40e6 / (2 * 112 * 111 * 336), "profiles/k_resid_ur_mixed_112x112x336_full.md"),
    # mean of the captured r, theta and phi solves of T (non-final, non-final, final)
    (True, "solve"): ((185.524e6 + 182.543e6 + 190.098e6) / (3 * 2 * 112 * 112 * 336),
                      "profiles/line_kernels_mixed_112x112x336_full.md"),
}


def max_over_ranks(value, dist, device):
    """Largest `value` over the ranks of the process group (all_reduce MAX); the
    value itself without one.  The job's time is the slowest rank's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, cells, steps, seconds):
    """Whole-job cell-updates/s: every rank advances its own shell (replicas,
    weak scaling), the job takes the slowest rank's time."""
    return world * cells * steps / seconds


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (background)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm = [float(r[1]) for r in rows if len(r) >= 9]
        mx = [float(r[2]) for r in rows if len(r) >= 9]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def workload(n, dt=5e-4, K=3):
    return dict(R1=0.5, R2=1.0, Pr=1.0, Ra=1e3, Nr=n, Nth=n, Nph=3 * n, dt=dt), K


def inputs(kw):
    from paper_1905_02300_gb300 import workloads as W
    spec = W.Spec(kw["R1"], kw["R2"], kw["Nr"], kw["Nth"], kw["Nph"], r_half=kw.get("r_half"))
    ex = W.TrigShell(kw["R1"], kw["R2"], kw["Pr"], kw["Ra"])
    return (W.sample_fields(ex, spec, 0.0), W.sample_fields(ex, spec, -kw["dt"]), W.forcing_modes(ex, spec))


def oracle_sample(n, K, steps):
    """Time the FP64 oracle for `steps` AC steps on an n x n x 3n shell."""
    from oracle.scheme import Oracle, Params
    kw, _ = workload(n)
    f0, fm, modes = inputs(kw)
    o = Oracle(Params(**kw))
    for lvl, f in ((0, f0), (1, fm)):
        o.set_fields(lvl, f["T"], f["ur"], f["uth"], f["uph"], f["p"])
    for tid, F in modes:
        o.set_forcing(tid, F["T"], F["ur"], F["uth"], F["uph"])
    t0 = time.perf_counter()
    o.step(steps, K)
    el = time.perf_counter() - t0
    cells = 2 * n * n * 3 * n
    return cells * steps / el, el


def ensemble_shells(seed, n, nr_max, nth_max, ys, precision):
    """Seeded uneven shells (workloads.shell_ensemble): convection start with a
    hot inner wall and the perturbation of wave numbers k, l, m <= 6,
    dt = 0.5 h_min^2 min(1, sqrt(1e3 / Ra)) per shell, h_min the smallest of
    h_r, R1 h_theta and R1 sin(theta_1) h_phi: inside the fixed-iteration
    stability limit dt < chi h^2, and short enough at high Ra that a run of
    a few hundred steps stays in the growth phase of the convection (its
    growth rate rises like sqrt(Ra); the saturated flow at Ra ~ 1e6 would
    need an advective CFL limit near 1e-6, and with 0.5 h_min^2 alone some
    shells of the ensemble overflow within 100 steps)."""
    from paper_1905_02300_gb300 import workloads as W
    out = []
    for idx, sp in enumerate(W.shell_ensemble(seed=seed, n=n, nr_max=nr_max, nth_max=nth_max)):
        spec = W.Spec(sp["R1"], sp["R2"], sp["Nr"], sp["Nth"], sp["Nph"])
        hmin = min(spec.hr, sp["R1"] * spec.hth, sp["R1"] * math.sin(spec.th0) * spec.hph)
        kw = dict(R1=sp["R1"], R2=sp["R2"], Pr=sp["Pr"], Ra=sp["Ra"], Nr=sp["Nr"], Nth=sp["Nth"], Nph=sp["Nph"],
                  dt=0.5 * hmin * hmin * min(1.0, math.sqrt(1e3 / sp["Ra"])), T_inner=1.0, T_outer=0.0,
                  precision=precision)
        out.append((kw, lambda spec=spec, sp=sp, idx=idx: W.convection_initial(spec, sp["Pr"], sp["Ra"],
                                                                                 seed=seed + idx, kmax=6)))
    return out


def class_roofline(prof, cells, mixed, hbm, src):
    """Roofline figures per kernel class from live CUDA-event tallies
    {class: (ms, launches)}: algorithmic bytes per launch = WORDS_PER_CELL x
    the cells one launch processes; the three line-solve classes are one
    kernel family (the line solves)."""
    merged = {}
    for k, (t_ms, n_l) in prof.items():
        key = "solve" if k.startswith("sweep_") else k
        w = WORDS_PER_CELL.get(k)
        b = ((w[0] * (4.0 if mixed else 8.0) + w[1] * 8.0) * cells * n_l) if w is not None else 0.0
        m = merged.setdefault(key, [0.0, 0, 0.0, 0.0])
        m[0] += t_ms
        m[1] += n_l
        m[2] += b
        m[3] += (0.0 if mixed else FLOPS_PER_CELL.get(k, 0.0)) * cells * n_l
    total = sum(v[0] for v in prof.values())
    out = {}
    for k, (t_ms, n_l, by, fl) in merged.items():
        if not n_l or not t_ms:
            continue
        gbs = by / (t_ms * 1e-3) / 1e9
        out[k] = {"ms": t_ms, "launches": n_l, "share": t_ms / total, "gbs": gbs, "hbm_frac": gbs / hbm,
                  "tflops": fl / (t_ms * 1e-3) / 1e12, "bytes_per_launch": by / n_l}
    return out


def run_ensemble(args):
    """Ensemble workload (the uneven-shell ensemble: 64 seeded shells, Nr
    16-64, Nth 16-96, Nph = 3 Nth): one batch, one launch per kernel class,
    one CUDA graph per step, autotuned lines per block, mixed precision, 100
    timed steps; per-class CUDA-event times from 2 further steps launched
    eagerly (ys_batch_profile_*); against the plain single-shell FP64 path
    running the same shells one at a time."""
    import torch
    from paper_1905_02300_gb300 import ys
    shells = ensemble_shells(4, args.ensemble_shells, 64, 96, ys, ys.YS_MIXED)
    cells = sum(2 * kw["Nr"] * kw["Nth"] * kw["Nph"] for kw, _ in shells)
    b = ys.Batch(len(shells), precision=ys.YS_MIXED, n_schwarz=3)
    for kw, init in shells:
        s = ys.Solver(**kw)
        s.set_fields_dict(0, init())
        b.add(s)
    chosen = b.autotune(trial_steps=2)
    b.step(max(args.warmup, 3))
    b.sync()
    steps = args.ensemble_steps
    st = torch.cuda.ExternalStream(b.stream_handle())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    time.sleep(0.3)
    e0.record(st)
    b.step(steps)
    e1.record(st)
    b.sync()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    value = cells * steps / (ms / 1e3)
    nrm = np.empty(ys.NFIELDS)
    diverged = sum(ys.lib.ys_batch_norms(b.h, slot, ys._ptr(nrm)) != ys.YS_OK for slot in list(b.members))
    b.profile(True)
    b.step(2)
    prof = b.profile_read()
    b.profile(False)
    hbm, src = peaks()
    cr = class_roofline(prof, cells, True, hbm, src)
    top = max(cr, key=lambda k: cr[k]["ms"])
    roof = {"bound": "hbm", "achieved": cr[top]["gbs"], "peak": hbm, "unit": "GB/s", "frac": cr[top]["hbm_frac"],
            "traffic": None, "kernel": top, "peak_source": src, "kernel_share": cr[top]["share"],
            "note": f"batched launches over all {len(shells)} shells; per-class times from 2 eagerly launched steps"}
    lps = b.launches_per_step()
    b.close()
    # plain FP64 single-shell path, one shell at a time, same shells
    t_fp64 = 0.0
    n64 = args.steps
    for kw, init in shells:
        s = ys.Solver(**dict(kw, precision=ys.YS_FP64))
        s.set_fields_dict(0, init())
        s.step(1, 3)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        sst = torch.cuda.Stream()
        s.set_stream(sst.cuda_stream)
        ev[0].record(sst)
        s.step(n64, 3)
        ev[1].record(sst)
        torch.cuda.synchronize()
        t_fp64 += ev[0].elapsed_time(ev[1]) / 1e3
        s.close()
    fp64_value = cells * n64 / t_fp64
    return {"metric": METRIC, "value": value, "unit": UNIT, "steps": steps, "ms_per_step": ms / steps,
            "dtype": "f32+f64", "members_diverged": int(diverged), "clocks": clk, "roofline": roof,
            "line_solves": cr.get("solve"),
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "config": {"workload": f"ensemble of {len(shells)} seeded uneven shells (Nr 16-64, Nth 16-96, "
                                   f"Nph=3Nth, R1/R2 0.35-0.6, Ra 1e3-1e6, Pr 0.7/1/7, perturbation k,l,m<=6), "
                                   f"K=3, mixed FP32/FP64, one batched launch per kernel class, CUDA graph per step",
                       "cells_total": cells, "lines_per_block": chosen, "launches_per_step": lps},
            "plain_fp64_one_at_a_time": {"value": fp64_value, "unit": UNIT, "steps": n64},
            "speedup_vs_plain_fp64": value / fp64_value}


def run_serving(args):
    """Serving workload: Poisson arrivals (seed 5) of shell simulations from the
    uneven-shell distribution extended to Nr <= 128 and Nth <= 192 (Nph up to
    576), N ~ U{50..500} steps each, at 0.8 of the measured batched capacity;
    p50/p99 time from submission to completion and aggregate cell-updates/s,
    with SM clocks sampled during the trace.  Against the same trace served
    FIFO one at a time by the plain FP64 path, whose run time per request is
    modelled as N (a + b cells) from FP64 steps timed on shells spanning the
    size range."""
    import torch
    from paper_1905_02300_gb300 import ys
    rng = np.random.default_rng(5)
    R = args.requests
    shells = ensemble_shells(5, R, 128, 192, ys, ys.YS_MIXED)
    steps = [int(rng.integers(50, 501)) for _ in range(R)]
    sizes = [2 * kw["Nr"] * kw["Nth"] * kw["Nph"] for kw, _ in shells]
    work = [c * n for c, n in zip(sizes, steps)]
    # initial states, built on the host cores in parallel (numpy releases the
    # interpreter lock in its array kernels) ahead of the arrivals: the
    # first 16 before the capacity probe, the rest while the trace runs
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(max(1, min(16, len(os.sched_getaffinity(0)))))
    futs = [pool.submit(sh[1]) for sh in shells]
    order = np.argsort(sizes)
    probe = [int(order[k]) for k in np.linspace(0, R - 1, 6).round().astype(int)]
    kept = {}
    # batched capacity from a short batch of the first 16 shells
    b = ys.Batch(16, precision=ys.YS_MIXED, n_schwarz=3)
    for (kw, _), fu in zip(shells[:16], futs[:16]):
        s = ys.Solver(**kw)
        s.set_fields_dict(0, fu.result())
        b.add(s)
    b.step(2)
    b.sync()
    t0 = time.perf_counter()
    b.step(5)
    b.sync()
    cap = sum(sizes[:16]) * 5 / (time.perf_counter() - t0)
    b.close()
    lam = 0.8 * cap / float(np.mean(work))           # requests per second
    arrivals = np.cumsum(rng.exponential(1.0 / lam, size=R))
    srv = ys.Server(hbm_budget_bytes=args.serving_budget_gb << 30, max_slots=R)
    tickets = [None] * R
    done = {}
    lag = 0.0
    clocks = Clocks(0)
    clocks.start()
    t_start = time.perf_counter()
    i = 0
    while len(done) < R:
        now = time.perf_counter() - t_start
        while i < R and arrivals[i] <= now:
            f0 = futs[i].result()
            lag = max(lag, time.perf_counter() - t_start - arrivals[i])
            tickets[i] = srv.submit(f0, steps[i], **shells[i][0])
            if i in probe:
                kept[i] = f0
            futs[i] = None
            i += 1
        for j in range(i):
            if j in done:
                continue
            st_, _, lat, rc = srv.poll(tickets[j], fields=False)
            if st_ >= 2:
                done[j] = (st_, lat, rc)
        time.sleep(0.001)
    wall = time.perf_counter() - t_start
    clk = clocks.stop()
    pool.shutdown()
    stats = srv.stats()
    srv.close()
    lats = np.array([done[j][1] for j in range(R)])
    ok = sum(1 for j in range(R) if done[j][0] == 2)
    # plain FP64 step time as a + b cells, fitted to shells across the size range
    pts = []
    for j in probe:
        s = ys.Solver(**dict(shells[j][0], precision=ys.YS_FP64))
        s.set_fields_dict(0, kept[j])
        s.step(1, 3)
        s.stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(3, 3)
        s.stats()
        pts.append((sizes[j], (time.perf_counter() - t0) / 3))
        s.close()
    A = np.array([[1.0, c] for c, _ in pts])
    coef = np.linalg.lstsq(A, np.array([t for _, t in pts]), rcond=None)[0]
    run_t = [n * max(coef[0] + coef[1] * c, 0.0) for c, n in zip(sizes, steps)]
    free_at, fifo_lat = 0.0, []
    for a, rt in zip(arrivals, run_t):
        start = max(a, free_at)
        free_at = start + rt
        fifo_lat.append(free_at - a)
    fifo_lat = np.array(fifo_lat)
    return {"metric": "served p50/p99 time to completion; cell-updates/s", "unit": "s",
            "value": float(np.percentile(lats, 50)), "p50_s": float(np.percentile(lats, 50)),
            "p99_s": float(np.percentile(lats, 99)), "higher_is_better": False,
            "requests": R, "completed": ok, "aggregate_cell_updates_per_s": float(sum(work) / wall),
            "trace_wall_s": wall, "arrival_rate_per_s": lam, "batched_capacity_estimate": cap,
            "submit_lag_max_s": lag,
            "clocks": clk, "dtype": "f32+f64",
            "fifo_plain_fp64": {"p50_s": float(np.percentile(fifo_lat, 50)),
                                "p99_s": float(np.percentile(fifo_lat, 99)),
                                "aggregate_cell_updates_per_s": float(sum(work) / max(free_at, arrivals[-1])),
                                "model": "per-request FP64 time N (a + b cells), a, b fitted to 3 timed FP64 "
                                         "steps of 6 shells across the size range",
                                "fit_s": [float(coef[0]), float(coef[1])]},
            "config": {"workload": f"{R} Poisson-arriving shells (seed 5) from the uneven-shell distribution "
                                   f"extended to Nr <= 128, Nth <= 192, Nph = 3 Nth; N in [50, 500] steps; K=3, "
                                   f"mixed FP32/FP64, continuous batching, lambda = 0.8 x batched capacity",
                       "cells_total_work": float(sum(work)), "hbm_budget_gb": args.serving_budget_gb},
            "server_steps": stats["steps"]}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    n = args.ref_n
    _, K = workload(args.n)
    for _ in range(args.warmup):
        oracle_sample(n, K, 1)
    v, el = oracle_sample(n, K, args.steps)
    cores = 1
    sample = f"{args.steps} AC step{'s' if args.steps != 1 else ''} of a {n}x{n}x{3*n}-per-patch shell (same physics, dt, K={K}) on 1 host core"
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"yin-yang shell {args.n}x{args.n}x{3*args.n} per patch, FP64, K=3 (sampled)",
                       "sample_grid": f"{n}x{n}x{3*n}"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_shell(args, mixed, dist=None, world=1, rank=0, local=0, with_cpu=True):
    """One Yin-Yang shell (the c2 / c3 grid 128 x 128 x 384 per patch, K = 3):
    device-timed cell-updates/s, e2e through the C ABI with pinned host
    buffers, per-class CUDA-event times and the roofline of the top class."""
    import torch
    from paper_1905_02300_gb300 import ys
    kw, K = workload(args.n)
    if args.stretch is not None:
        from paper_1905_02300_gb300 import workloads as W
        kw["r_half"] = W.stretched_radii(kw["R1"], kw["R2"], kw["Nr"], args.stretch)
    f0, fm, modes = inputs(kw)
    s = ys.Solver(**kw, precision=ys.YS_MIXED if mixed else ys.YS_FP64)
    stream = torch.cuda.Stream()
    s.set_stream(stream.cuda_stream)
    s.set_fields_dict(0, f0)
    s.set_fields_dict(1, fm)
    for m, (tid, F) in enumerate(modes):
        s.set_forcing(m, tid, F["T"], F["ur"], F["uth"], F["uph"])
    cells = 2 * kw["Nr"] * kw["Nth"] * kw["Nph"]

    s.step(args.warmup, K)
    torch.cuda.synchronize()
    # the FP64 pipe's own rate on this device, the denominator of the FP64
    # form's ALU-bound kernels (median of 3 probes)
    fp64_peak = statistics.median(ys.measure_fp64_rate() for _ in range(3))
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.4)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    s.profile(True)
    n_launch0 = s.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(args.steps, K)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = s.launch_count() - n_launch0
    prof = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = job_throughput(world, cells, args.steps, ms_max / 1e3)

    # end to end through the C ABI with pinned host buffers
    pinned = {}
    for lvl, f in ((0, f0), (1, fm)):
        for k, a in f.items():
            t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = a
            pinned[(lvl, k)] = t.numpy()
    out = {k: torch.empty(a.shape, dtype=torch.float64, pin_memory=True).numpy() for k, a in f0.items()}
    h2d = 2 * sum(a.nbytes for a in f0.values())
    d2h = sum(a.nbytes for a in f0.values())
    t_e2e = []
    for it in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for lvl in (0, 1):
            s.set_fields(lvl, *[pinned[(lvl, k)] for k in ("T", "ur", "uth", "uph", "p")])
        s.step(1, K)
        rc = ys.lib.ys_get_fields(s.h, 0, *[ys._ptr(out[k]) for k in ("T", "ur", "uth", "uph", "p")], None)
        if rc:
            raise ys.YSError(rc, "ys_get_fields")
        if it > 0:
            t_e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(statistics.median(t_e2e), dist, "cuda")
    e2e_val = job_throughput(world, cells, 1, e2e_s)
    state_gb = s.device_bytes() / 1e9
    s.close()

    # roofline of the dominant kernel class (the three line-solve classes are
    # one kernel family)
    hbm, src = peaks()
    cr = class_roofline(prof, cells, mixed, hbm, src)
    top = max(cr, key=lambda k: cr[k]["ms"])
    c = cr[top]
    if c["tflops"] and c["tflops"] / fp64_peak > c["hbm_frac"]:
        roof = {"bound": "alu", "achieved": c["tflops"], "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": c["tflops"] / fp64_peak, "traffic": None, "kernel": top,
                "peak_source": "measured in this run: ys_measure_fp64_rate (independent FP64 FMA chains on "
                               "every SM, CUDA events); nominal %.2f" % FP64_PEAK_TFLOPS,
                "hbm_gbs": c["gbs"], "hbm_frac": c["hbm_frac"]}
    else:
        roof = {"bound": "hbm", "achieved": c["gbs"], "peak": hbm, "unit": "GB/s", "frac": c["hbm_frac"],
                "traffic": None, "kernel": top, "peak_source": src}
    roof["kernel_share"] = c["share"]
    roof["launches"] = c["launches"]
    tp = TRAFFIC_PER_POINT.get((mixed, top))
    if tp is not None:
        roof["traffic"] = tp[0] * cells
        roof["traffic_source"] = tp[1] + " (scaled from the capture's points to this launch)"
    roof["algorithmic_bytes_per_launch"] = c["bytes_per_launch"]

    cpu = None
    if rank == 0 and with_cpu and not args.no_cpu_baseline:
        v, el = oracle_sample(args.ref_n, K, args.ref_steps)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{args.ref_steps} AC steps (K={K}) of a {args.ref_n}x{args.ref_n}x{3*args.ref_n}-per-patch "
                         f"shell, same physics and dt, numpy on 1 host core, {el:.1f} s"}
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if mixed else "f64",
            "data": "synthetic",
            "config": {"workload": f"yin-yang shell {args.n}x{args.n}x{3*args.n} MAC cells per patch, "
                                   f"R1=0.5 R2=1 Pr=1 Ra=1e3 dt=5e-4, K={K} Schwarz iterations, "
                                   f"{'mixed FP32/FP64' if mixed else 'FP64'}, "
                                   f"manufactured-solution forcing"
                                   + (f", stretched radial grid (beta {args.stretch})"
                                      if args.stretch is not None else ""),
                       "cells_per_shell": cells, "l2": "inputs larger than L2 (state ~%.1f GB)" % state_gb,
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "fp64_peak_tflops_measured": fp64_peak,
            "line_solves": cr.get("solve"),
            "kernels_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "kernels_launches": {k: v[1] for k, v in prof.items() if v[1]}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--ref-n", type=int, default=48)
    ap.add_argument("--ref-steps", type=int, default=8, help="oracle steps of the cpu_baseline sample (~12 s)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stretch", type=float, default=None,
                    help="run the shell on a stretched radial grid (workloads.stretched_radii beta)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--workload", default="all", choices=["all", "shell", "ensemble", "serving"],
                    help="all (default): the FP64 shell line with the mixed, ensemble and serving results "
                         "as objects of the same line (one GPU only)")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--ensemble-shells", type=int, default=64,
                    help="shells of the ensemble workload (64 as specified; fewer for a short profiling case)")
    ap.add_argument("--serving-budget-gb", type=int, default=200)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = env_rank()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (the product path has no CPU fallback)")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    if args.workload in ("ensemble", "serving"):
        line = (run_ensemble if args.workload == "ensemble" else run_serving)(args)
        print(json.dumps(line), flush=True)
        return 0

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = run_shell(args, args.precision == "mixed", dist, world, rank, local)
    if args.workload == "all" and world == 1:
        t0 = time.perf_counter()
        m = run_shell(args, True, with_cpu=False)
        line["mixed"] = {k: m[k] for k in ("value", "unit", "ms_per_step", "dtype", "e2e", "roofline", "line_solves",
                                           "clocks", "gpu_launches", "kernels_ms")}
        line["mixed"]["config"] = m["config"]["workload"]
        line["ensemble"] = run_ensemble(args)
        line["serving"] = run_serving(args)
        line["config"]["also"] = ("mixed (same shell, FP32 bulk), ensemble (64 uneven shells, batched), "
                                  "serving (200 Poisson-arriving requests): objects of this line, %.0f s"
                                  % (time.perf_counter() - t0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
