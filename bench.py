#!/usr/bin/env python
"""Benchmark of the B300 bootstrap particle filter.

Default workload: Lorenz '96, N=40, F=8, RK4 dt=0.005 x 10 substeps per
observation, every 2nd component observed with N(0,1) noise, P=2^20
particles, T=500 observations, FP32 propagation / FP64 weights (the Large
configuration).  One step = one whole filter run (all T observations:
propagate, weight, log-sum-exp, ESS test, systematic resampling) over one
synthetic observation series; the metric is particle-steps/s (P*T per run).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: one process per GPU (torchrun); every rank runs an independent
filter replica (different seed), no collective on the data path; value = all
ranks' particle-steps / max-over-ranks time ("weak" scaling).

--impl reference times the CPU oracle (plain C, OpenMP over particles) on the
host cores on a bounded sample of the same workload.
"""
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")
SERVER_BRANCHES = 4  # concurrent launch groups per server iteration (the library default)
DESCRIPTOR_BYTES = 272  # per-filter descriptor the library uploads with every run


def _code_only(text):
    """Source text without // comments, trailing blanks and empty lines, so the
    hash below changes with the code of the kernels and not with their comments."""
    out = []
    for line in text.splitlines():
        k = line.find("//")
        if k >= 0:
            line = line[:k]
        line = line.rstrip()
        if line:
            out.append(line)
    return "\n".join(out)


def kernel_source_hash(read=None):
    """Hash of the code of pf_kernels.cu and pf_dev.cuh (comments ignored)."""
    h = hashlib.sha256()
    for fn in ("pf_kernels.cu", "pf_dev.cuh"):
        if read is None:
            with open(os.path.join(ROOT, "paper_1306_3277_b300", "csrc", fn)) as f:
                text = f.read()
        else:
            text = read(fn)
        h.update(_code_only(text).encode())
    return h.hexdigest()[:16]


def read_traffic(kernel_tag, P):
    """Per-launch DRAM bytes of a kernel from its committed ncu summary, if the
    summary was taken on the current kernel source and at this particle count
    (else None)."""
    path = os.path.join(PROFILES, "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(kernel_tag)
    if not e or e.get("kernel_source_hash") != kernel_source_hash() or e.get("P") != P:
        return None
    return e.get("dram_bytes_per_launch")


L2_BYTES = 126 << 20


def l2_note(w):
    """How the timed region stands to the 126 MB L2 (no flush is done: the
    headline state streams from HBM every step; small filters are L2-resident
    and latency-bound by design)."""
    state = w.N * w.P * (4 if w.prec else 8)
    if 2 * state > L2_BYTES:
        return "inputs larger than L2 (state %d MiB x 2)" % (state >> 20)
    return ("L2-resident working set (state %.1f KiB x 2), not flushed: a latency-bound "
            "configuration" % (state / 1024.0))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)
        if not self.rows:
            return None

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in self.rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in self.rows) if v is not None]
        pw = [v for v in (num(r[3]) for r in self.rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": reasons,
                "samples": len(self.rows)}


def l96_flops_per_particle_step(w):
    """Algorithmic FP32 flops of one Lorenz '96 particle-step: RK4 (4
    right-hand sides of 2 sub + 1 fma = 4 flop, 3 stage fmas, 4 combination
    fmas = 30 flop per component and substep) plus the noise fma (2 flop per
    component).  Random-number generation is not counted."""
    return 30 * w.N * w.substeps + 2 * w.N


def propagate_bytes_per_particle(w):
    """Algorithmic HBM bytes of the propagate kernel per particle: ancestor
    read (4), state gather read and write (2 N sizeof), in-tile weight prefix
    write (8)."""
    sb = 4 if w.prec == W.MIXED else 8
    return 2 * w.N * sb + 12


RESAMPLE_BYTES_PER_PARTICLE = 12  # weight prefix read (8) + ancestor write (4)


def make_workload(args):
    if args.config == "large":
        return W.lorenz96_large(P=args.P or (1 << 20), T=args.T or 500)
    if args.config == "l96_8":
        return W.lorenz96_8(P=args.P or (1 << 14), T=args.T or 200, prec=W.MIXED)
    if args.config == "l96_8_fp64":
        return W.lorenz96_8(P=args.P or (1 << 14), T=args.T or 200, prec=W.FP64)
    if args.config == "windkessel_mixed":
        return W.windkessel(P=args.P or 1024, T=args.T or 100, prec=W.MIXED)
    return W.windkessel(P=args.P or 1024, T=args.T or 100)


def cpu_oracle_rate(w, P_sample, T_sample, nthreads=0, min_secs=0.0):
    """Particle-steps/s of the oracle on a bounded sample of workload w.

    A sample shorter than min_secs of wall time is run again with the next seeds until it is
    not (a whole small filter takes milliseconds); the rate covers every run.
    Returns (rate, seconds, runs)."""
    import oracle as O
    ws = w.with_(P=P_sample, T=T_sample, y=w.y[:T_sample].copy())
    m = O.model(ws.kind, N=ws.N, substeps=ws.substeps, obs_stride=ws.obs_stride, prec=ws.prec,
                dt=ws.dt, ess_threshold=ws.ess_threshold, flow_peak=ws.flow_peak,
                flow_period=ws.flow_period)
    runs = 0
    t0 = time.perf_counter()
    while True:
        O.pf_run(m, ws.theta, ws.y, 1 + runs, ws.P, ws.T, nthreads=nthreads, want_x=False,
                 want_anc=False, want_diag=False)
        runs += 1
        dt = time.perf_counter() - t0
        if dt >= min_secs or runs >= 100000:
            break
    return ws.P * ws.T * runs / dt, dt, runs


def oracle_sample(w):
    """Sample sizes for the oracle: about 10 s of CPU work on 16 cores."""
    if w.kind == W.LORENZ96 and w.N >= 40:
        return min(w.P, 1 << 18), min(w.T, 40)
    if w.kind == W.LORENZ96:
        return min(w.P, 1 << 14), min(w.T, 100)
    return min(w.P, 1 << 14), min(w.T, 100)


def cores():
    return len(os.sched_getaffinity(0))


def max_over_ranks(x, dist=None, device=None):
    """The largest of every rank's value (the whole job ends with its slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(units_per_rank, world, elapsed_s):
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return units_per_rank * world / elapsed_s


def dtype_name(w):
    return "f64" if w.prec == W.FP64 else "f32 state / f64 weights"


def run_reference(args):
    """The CPU oracle as it stands, on the host cores, bounded samples."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    w = make_workload(args)
    P_s, T_s = oracle_sample(w)
    P_s = max(P_s // 4, 1)  # a quarter of the baseline sample per step: K steps stay short
    for _ in range(args.warmup):
        cpu_oracle_rate(w, max(P_s // 16, 1), 1)
    secs = []
    for _ in range(args.steps):
        secs.append(cpu_oracle_rate(w, P_s, T_s)[1])
    total = sum(secs)
    value = P_s * T_s * args.steps / total
    sample = "P=%d T=%d of %s per step, OpenMP over particles" % (P_s, T_s, w.name)
    line = {"impl": "reference", "metric": "particle-steps/s", "value": value,
            "unit": "particle-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_name(w), "data": "synthetic",
            "config": {"workload": w.name, "P": w.P, "T": w.T, "N": w.N,
                       "substeps": w.substeps, "obs_stride": w.obs_stride},
            "cpu_baseline": {"value": value, "unit": "particle-steps/s", "cores": cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def secondary(pf, torch, dev):
    """Quick extra numbers: the small configurations and batched vs plain."""
    out = {}
    st = torch.cuda.Stream(device=dev)

    def time_runs(w, reps):
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        th = torch.tensor(w.theta, dtype=torch.float64, device=dev)
        y = torch.tensor(w.y, dtype=torch.float64, device=dev)
        ll = torch.zeros(1, dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        for r in range(3):
            pf.pf_run(f, th, y, 100 + r, ll, None, None, pf.PF_FLAG_ASYNC, st)
        st.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for r in range(reps):
            pf.pf_run(f, th, y, r + 1, ll, None, None, pf.PF_FLAG_ASYNC, st)
        e1.record(st)
        st.synchronize()
        ms = e0.elapsed_time(e1) / reps
        f.destroy()
        return ms

    for name, w, reps in (("windkessel_P1024_T100_fp64", W.windkessel(), 50),
                          ("lorenz96_N8_P16384_T200_fp64", W.lorenz96_8(), 10),
                          ("lorenz96_N8_P16384_T200_mixed", W.lorenz96_8(prec=W.MIXED), 10)):
        ms = time_runs(w, reps)
        out[name] = {"ms_per_run": ms, "particle_steps_per_s": w.P * w.T / (ms * 1e-3),
                     "runs_per_s": 1e3 / ms}
    # batched: 256 uneven filters in one plan (CUDA graph) vs one pf_run per filter
    ws = W.batched()
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    ths = [w.theta for w in ws]
    ys = [w.y for w in ws]
    seeds = [w.seed for w in ws]
    pf.pf_batch_run(fs, ths, ys, seeds)  # plan + graph build
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        lls_b, _ = pf.pf_batch_run(fs, ths, ys, seeds)
    tb = (time.perf_counter() - t0) / reps
    for f, w in zip(fs, ws):  # build the single-filter plans
        f.run(w.theta, w.y, w.seed)
    t0 = time.perf_counter()
    lls_p = [f.run(w.theta, w.y, w.seed)[1] for f, w in zip(fs, ws)]
    tp = time.perf_counter() - t0
    maxrel = max(abs(a - b) / abs(b) for a, b in zip(lls_b, lls_p))
    psteps = sum(w.P * w.T for w in ws)
    # the autotuned launch shape: cluster bound, branches, resample grid
    chosen = pf.pf_batch_autotune(fs, ths, ys, seeds)
    shape = pf.pf_batch_get_shape(fs)
    pf.pf_batch_run(fs, ths, ys, seeds)  # the chosen shape's plan and graph
    t0 = time.perf_counter()
    for _ in range(reps):
        lls_a, _ = pf.pf_batch_run(fs, ths, ys, seeds)
    ta = (time.perf_counter() - t0) / reps
    maxrel_a = max(abs(a - b) / abs(b) for a, b in zip(lls_a, lls_p))

    def batch_ms(cta, branches, rs, persistent=0, kt=1):
        pf.pf_batch_set_shape(fs, cta, branches, rs, persistent, kt)
        pf.pf_batch_run(fs, ths, ys, seeds)  # plan + graph build
        t0 = time.perf_counter()
        for _ in range(reps):
            pf.pf_batch_run(fs, ths, ys, seeds)
        return (time.perf_counter() - t0) / reps * 1e3

    # the batch at candidate shapes (one field at a time, as the autotuner searches)
    sweep_cta = {str(b): batch_ms(b, 1, 8) for b in (0, 256, 1024, 2048)}
    sweep_br = {str(k): batch_ms(0, k, 8) for k in (1, 2, 4, 8, 16)}
    # the persistent launch: CTAs per SM x tiles per propagate item
    sweep_pe = {"%d_%d" % (b, kt): batch_ms(0, 1, 8, b, kt)
                for b, kt in ((2, 1), (3, 1), (4, 1), (4, 2), (4, 4))}
    pf.pf_batch_set_shape(fs, shape["cta_max_particles"], shape["branches"],
                          shape["resample_blocks_per_sm"], shape["persistent_blocks_per_sm"],
                          shape["tiles_per_item"])
    out["batched_256"] = {"filters": len(ws), "batched_evals_per_s": len(ws) / tb,
                          "plain_evals_per_s": len(ws) / tp, "speedup": tp / tb,
                          "batched_particle_steps_per_s": psteps / tb,
                          "max_rel_loglik_diff_vs_plain": maxrel,
                          "autotuned_shape": shape,
                          "autotuned_cluster_max_particles": chosen,
                          "autotuned_evals_per_s": len(ws) / ta,
                          "autotuned_speedup_vs_plain": tp / ta,
                          "autotuned_max_rel_loglik_diff_vs_plain": maxrel_a,
                          "batch_ms_by_cluster_bound": sweep_cta,
                          "batch_ms_by_branches": sweep_br,
                          "batch_ms_persistent_by_ctas_per_sm_and_tiles_per_item": sweep_pe}
    for f in fs:
        f.destroy()
    # one small filter alone: the tiled launches against one cluster per filter
    for w in (W.windkessel(P=1024, T=100, prec=W.MIXED),
              W.lorenz96_8(P=1024, T=200, prec=W.MIXED)):
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        small = {}
        for name, cta in (("tiled", 0), ("cluster", 4096)):
            pf.pf_batch_configure([f], cta)
            pf.pf_batch_run([f], [w.theta], [w.y], [w.seed])
            t0 = time.perf_counter()
            for _ in range(20):
                pf.pf_batch_run([f], [w.theta], [w.y], [w.seed])
            small[name + "_ms_per_run"] = (time.perf_counter() - t0) / 20 * 1e3
        f.destroy()
        out["small_filter_" + w.name] = small
    # serving: the rate sweep up to the stated 2000 requests/s (10 s of Poisson
    # arrivals per rate, so 20,000 requests at the top rate, then at most 5 s
    # more to drain; an overloaded rate reports its unfinished requests),
    # beside the same request mix one pf_run at a time
    fp32_peak = pf.pf_measure_fma_peak(pf.PF_MIXED)
    serving = {"arrivals_s": 10.0, "drain_s": 5.0,
               "rates": [serve_at_rate(pf, rate, 10.0, 5.0, 64 << 30, 128, fp32_peak,
                                       SERVER_BRANCHES)
                         for rate in (250.0, 500.0, 1000.0, 1500.0, 2000.0)]}
    reqs = W.serving_requests(40, 100.0, seed=7)
    fs = [(pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt), w) for _, w in reqs]
    for f, w in fs[:3]:
        f.run(w.theta, w.y, w.seed)
    t0 = time.perf_counter()
    for f, w in fs:
        f.run(w.theta, w.y, w.seed)
    serving["plain_requests_per_s"] = len(fs) / (time.perf_counter() - t0)
    for f, _ in fs:
        f.destroy()
    out["serving"] = serving
    return out


def request_flops(w):
    """Algorithmic FP32 flops of one served request (Lorenz '96 RK4 and noise;
    the windkessel's few FP64 operations are not counted)."""
    if w.kind == W.LORENZ96:
        return l96_flops_per_particle_step(w) * w.P * w.T
    return 0


def serve_at_rate(pf, rate, duration, drain, budget_bytes, slots, fp32_peak=None,
                  branches=None):
    """Poisson arrivals at `rate` per second for `duration` seconds into one
    server, then up to `drain` seconds for the queue to empty: goodput,
    latency quantiles of the completed requests, queue length (sampled every
    10 ms), rejected and unfinished requests."""
    n = max(1, int(rate * duration))
    reqs = W.serving_requests(n, rate, seed=int(rate))
    srv = pf.pf_server_create(budget_bytes, slots, branches=branches)
    pending = {}
    lat = []
    psteps_done = flops_done = 0
    rejected, max_queued, queued_at_end, last_stat = 0, 0, None, -1.0
    t0 = time.perf_counter()
    k = 0
    while k < len(reqs) or pending:
        now = time.perf_counter() - t0
        while k < len(reqs) and reqs[k][0] <= now:
            w = reqs[k][1]
            try:
                t = srv.submit(pf.model_from_workload(w), w.P, w.T, w.dt, w.theta, w.y, w.seed)
                pending[t] = w
            except pf.PFError:
                rejected += 1
            k += 1
        if now - last_stat >= 0.01:  # queue length, sampled every 10 ms
            queued = srv.stats()["queued"]
            max_queued = max(max_queued, queued)
            if queued_at_end is None and k == len(reqs):
                queued_at_end = queued
            last_stat = now
        for t in list(pending):
            r = srv.poll(t)
            if r is not None:
                w = pending.pop(t)
                lat.append(r[2])
                psteps_done += w.P * w.T
                flops_done += request_flops(w)
        if now > duration + drain:
            break
        time.sleep(0.0005)
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.destroy()
    lat.sort()
    q = (lambda f: lat[min(len(lat) - 1, int(f * len(lat)))] if lat else None)
    out = {"offered_per_s": rate, "submitted": k, "rejected": rejected, "completed": len(lat),
           "unfinished": len(pending), "max_queued": max_queued,
           "queued_when_arrivals_end": queued_at_end, "goodput_per_s": len(lat) / elapsed,
           "particle_steps_per_s": psteps_done / elapsed, "p50_s": q(0.5), "p99_s": q(0.99),
           "elapsed_s": elapsed, "iterations": st["iterations"], "branches": branches,
           "fp32_tflops": flops_done / elapsed / 1e12}
    if fp32_peak:
        out["fp32_roof_frac"] = flops_done / elapsed / fp32_peak
    return out


def run_serving(args):
    """Continuous-batching server under Poisson arrivals: a rate sweep with
    goodput and p50/p99 latency per offered rate, and the plain form (one
    pf_run per request, back to back) on a sample of the same requests."""
    import torch
    import paper_1306_3277_b300 as pf
    torch.cuda.set_device(0)
    rates = [float(r) for r in args.rates.split(",")]
    fp32_peak = None if args.no_peak else pf.pf_measure_fma_peak(pf.PF_MIXED)
    sweep = []
    for rate in rates:
        sweep.append(serve_at_rate(pf, rate, args.duration, args.drain,
                                   int(args.budget_gb * (1 << 30)), args.slots, fp32_peak,
                                   args.server_branches))
        print(json.dumps({"rate": rate, **sweep[-1]}), file=sys.stderr, flush=True)
    # plain form: the same kind of requests one pf_run at a time
    reqs = W.serving_requests(args.plain_sample, 100.0, seed=7)
    fs = [(pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt), w) for _, w in reqs]
    for f, w in fs[:3]:
        f.run(w.theta, w.y, w.seed)
    t0 = time.perf_counter()
    for f, w in fs:
        f.run(w.theta, w.y, w.seed)
    tp = time.perf_counter() - t0
    for f, _ in fs:
        f.destroy()
    best = max(sweep, key=lambda d: d["goodput_per_s"])
    out = {"metric": "requests/s (goodput) and p50/p99 latency", "value": best["goodput_per_s"],
           "unit": "requests/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32 state / f64 weights", "data": "synthetic",
           "config": {"workload": "serving: Poisson arrivals, models windkessel / L96 N=8 / "
                                  "L96 N=40, P=2^U{10..16}, T~U{50..1000}",
                      "slots": args.slots, "launch_groups": args.server_branches,
                      "budget_gb": args.budget_gb,
                      "duration_s": args.duration, "drain_s": args.drain},
           "sweep": sweep,
           "plain_one_run_at_a_time": {"requests": len(fs), "requests_per_s": len(fs) / tp,
                                       "note": "same request mix, one pf_run per request"}}
    print(json.dumps(out), flush=True)
    return 0


def run_precision(args):
    """Mixed (FP32 state, FP64 weights) minus FP64 log-likelihood on the same
    seeds, per configuration: mean and standard error over seeds."""
    import torch
    import paper_1306_3277_b300 as pf
    torch.cuda.set_device(0)
    cfgs = [("windkessel_P1024_T100", lambda p: W.windkessel(prec=p), args.seeds),
            ("lorenz96_N8_P16384_T200", lambda p: W.lorenz96_8(prec=p), args.seeds),
            ("lorenz96_N40_P65536_T100", lambda p: W.lorenz96_large(P=1 << 16, T=100, prec=p),
             max(8, args.seeds // 4))]
    res = {}
    for name, make, nseed in cfgs:
        out = {}
        for prec in (W.FP64, W.MIXED):
            w = make(prec)
            f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
            out[prec] = np.array([f.run(w.theta, w.y, s + 1)[1] for s in range(nseed)])
            f.destroy()
        d = out[W.MIXED] - out[W.FP64]
        res[name] = {"seeds": nseed, "mean_mixed_minus_fp64": float(d.mean()),
                     "se": float(d.std(ddof=1) / np.sqrt(nseed)),
                     "sd_fp64_over_seeds": float(out[W.FP64].std(ddof=1)),
                     "mean_fp64": float(out[W.FP64].mean())}
    print(json.dumps({"metric": "loglik(mixed) - loglik(fp64), same seeds", "results": res}),
          flush=True)
    return 0


def run_variants(args):
    """The Large shape (P = 2^20, N = 40, mixed) with each resampling scheme and
    the paper's stochastic Lorenz '96, plus the exact windkessel: ms per whole
    run (CUDA graph) and the per-step propagate / resample kernel times (one
    profiled run, events around every launch)."""
    import torch
    import paper_1306_3277_b300 as pf
    torch.cuda.set_device(0)
    T = args.T or 100
    large = W.lorenz96_large(T=T)
    cases = [("systematic", large), ("stratified", large.with_(resampler=1)),
             ("multinomial", large.with_(resampler=2)),
             ("sde_lorenz96", W.lorenz96_sde(P=1 << 20, T=T, N=40, substeps=10, dt=0.005,
                                             obs_stride=2, prec=W.MIXED,
                                             theta=(8.0, 0.01, 1.0, 0.0, 1.0))),
             ("sparse_every2_first10", W.lorenz96_large(T=T).with_(obs_every=2, obs_count=10)),
             ("one_rk4_substep", large.with_(substeps=1)),
             ("exact_windkessel_P1M", W.windkessel_exact(P=1 << 20, T=T, prec=W.MIXED))]
    out = {}
    for name, w in cases:
        if name == "sparse_every2_first10":
            w.y = W.simulate(w)
        f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
        for k in range(3):
            st, ll, _, _ = f.run(w.theta, w.y, 10 + k)
        t0 = time.perf_counter()
        reps = 3
        for k in range(reps):
            f.run(w.theta, w.y, 20 + k)
        ms = (time.perf_counter() - t0) / reps * 1e3
        pf.pf_profile_enable(f, True)
        f.run(w.theta, w.y, 30)
        prof = pf.pf_profile_read(f)
        pf.pf_profile_enable(f, False)
        f.destroy()
        pm, pn = prof["propagate"]
        rm, rn = prof["resample"]
        out[name] = {"P": w.P, "T": w.T, "ms_per_run": ms,
                     "particle_steps_per_s": w.P * w.T / (ms * 1e-3),
                     "propagate_ms_per_step": pm / max(pn, 1),
                     "resample_ms_per_step": rm / max(w.T - 1, 1),
                     "status": st, "loglik": ll}
        if name == "one_rk4_substep":
            # the step's algorithmic bytes (gather, write, weights, ancestors) over
            # its propagate + resample time, against the measured copy bandwidth
            step_bytes = (propagate_bytes_per_particle(w) + RESAMPLE_BYTES_PER_PARTICLE) * w.P
            step_s = (pm / max(pn, 1) + rm / max(w.T - 1, 1)) * 1e-3
            hbm = measured_peaks()[0]["hbm_gbs"]
            out[name]["step_bytes"] = step_bytes
            out[name]["step_hbm_gbs"] = step_bytes / step_s / 1e9
            out[name]["step_hbm_frac"] = step_bytes / step_s / 1e9 / hbm
    print(json.dumps({"metric": "ms per whole run, per-step kernel times", "results": out}),
          flush=True)
    return 0


def run_batched(args):
    """The batched form on its own: 256 uneven filters (Lorenz '96 N=8 and
    windkessel, P 2^8..2^14, T 50..500, mixed precision) as one plan, in the
    launch shape the autotuner picks (or, with --branches, that many launch
    chains, the small filters on thread-block clusters up to --cluster-bound
    particles, --rs-grid resample blocks per SM, and with --persistent that
    many CTAs per SM of the persistent launch, --tiles-per-item tiles per work
    item).  K timed batch runs after
    W warm-ups; unless --no-secondary, the same filters one pf_run at a time
    for comparison."""
    import torch
    import paper_1306_3277_b300 as pf
    torch.cuda.set_device(0)
    ws = W.batched()
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for w in ws]
    ths, ys, seeds = [w.theta for w in ws], [w.y for w in ws], [w.seed for w in ws]
    if args.branches > 0:
        pf.pf_batch_set_shape(fs, args.cluster_bound, args.branches, args.rs_grid,
                              args.persistent, args.tiles_per_item)
    else:
        pf.pf_batch_autotune(fs, ths, ys, seeds)
    shape = pf.pf_batch_get_shape(fs)
    for _ in range(max(args.warmup, 1)):  # the first run builds the plan and its graph
        pf.pf_batch_run(fs, ths, ys, seeds)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        lls, sts = pf.pf_batch_run(fs, ths, ys, seeds)
    tb = (time.perf_counter() - t0) / args.steps
    psteps = sum(w.P * w.T for w in ws)
    line = {"metric": "batched evaluations/s", "value": len(ws) / tb, "unit": "evals/s",
            "steps": args.steps, "warmup": max(args.warmup, 1), "ms_per_batch": tb * 1e3,
            "particle_steps_per_s": psteps / tb, "filters": len(ws),
            "shape": shape, "shape_from": "given" if args.branches > 0 else "autotuner",
            "degenerate": int(sum(1 for st in sts if int(st) != 0))}
    if not args.no_secondary:
        for f, w in zip(fs, ws):  # the single-filter plans
            f.run(w.theta, w.y, w.seed)
        t0 = time.perf_counter()
        lp = [f.run(w.theta, w.y, w.seed)[1] for f, w in zip(fs, ws)]
        tp = time.perf_counter() - t0
        line["plain_evals_per_s"] = len(ws) / tp
        line["speedup"] = tp / tb
        line["max_rel_loglik_diff_vs_plain"] = max(abs(a - b) / abs(b) for a, b in zip(lls, lp))
    for f in fs:
        f.destroy()
    print(json.dumps(line), flush=True)
    return 0


def run_samplers(args):
    """Throughput of the samplers built on the filter: marginal Metropolis-
    Hastings (64 chains, each iteration one batched launch of all chains'
    filters, split between the tiled and cluster paths by the autotuner) and
    SMC^2 (Algorithm 4, its O(T^2) rejuvenation runs included)."""
    import torch
    import paper_1306_3277_b300 as pf
    torch.cuda.set_device(0)
    inf = float("inf")
    out = {}
    w = W.windkessel(P=1024, T=100)
    spec = [(3, 1, 2.0, 0.9, 0.03, 0.0, inf), (0, 0), (3, 1, 2.0, 0.03, 0.002, 0.0, inf),
            (4, 2, 2.0, 0.01, 2.0, 3.0), (0, 0), (0, 0), (0, 0)]
    nc, niter = 64, 200
    fs = [pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt) for _ in range(nc)]
    th0 = np.tile(np.array(w.theta), (nc, 1))
    # the chains' filters form one batch: the autotuner picks its tiled / cluster split
    chosen = pf.pf_batch_autotune(fs, [w.theta] * nc, [w.y] * nc, list(range(1, nc + 1)))
    pf.pf_pmmh_run(fs, w.y, spec, th0, 5, 1)  # plan and graph
    t0 = time.perf_counter()
    _, _, acc = pf.pf_pmmh_run(fs, w.y, spec, th0, niter, 2)
    dt = time.perf_counter() - t0
    shape = pf.pf_batch_get_shape(fs)
    pf.pf_batch_set_shape(fs, 0, 1, 8, 0, 1)  # the same chains on one tiled launch chain
    pf.pf_pmmh_run(fs, w.y, spec, th0, 5, 1)
    t0 = time.perf_counter()
    pf.pf_pmmh_run(fs, w.y, spec, th0, niter, 2)
    dt_tiled = time.perf_counter() - t0
    for f in fs:
        f.destroy()
    out["pmmh_windkessel_P1024_T100_64chains"] = {
        "iterations": niter, "chains": nc, "seconds": dt,
        "chain_iterations_per_s": nc * (niter + 1) / dt,
        "particle_steps_per_s": nc * (niter + 1) * w.P * w.T / dt,
        "acceptance": float(acc.sum()) / (nc * niter),
        "autotuned_cluster_max_particles": chosen,
        "autotuned_shape": shape,
        "tiled_only_chain_iterations_per_s": nc * (niter + 1) / dt_tiled}
    w = W.windkessel(P=256, T=50)
    spec2 = [(0, 0), (0, 0), (3, 1, 2.0, 0.03, 0.005, 0.0, inf), (4, 2, 2.0, 0.01, 2.0, 3.0),
             (0, 0), (0, 0), (0, 0)]
    nt = 256
    m = pf.model_from_workload(w)
    pf.pf_smc2_run(m, w.P, 5, w.dt, w.y[:5], 8, spec2, w.theta, 1)  # warm the code path
    runs = []
    for _ in range(3):  # the median of three whole runs (each allocates its populations)
        t0 = time.perf_counter()
        st, th, logw, lz, incr, acc2 = pf.pf_smc2_run(m, w.P, w.T, w.dt, w.y, nt, spec2,
                                                      w.theta, 2)
        runs.append(time.perf_counter() - t0)
    dt = statistics.median(runs)
    steps = sum(2 * i - 1 for i in range(1, w.T + 1))  # rejuvenation runs + continuations
    out["smc2_windkessel_P256_T50_256theta"] = {
        "seconds": dt, "log_evidence": lz, "theta_particles": nt,
        "particle_steps_per_s": nt * steps * w.P / dt,
        "acceptance": float(acc2.sum()) / (nt * w.T)}
    print(json.dumps({"metric": "sampler throughput", "results": out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawTextHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large",
                    choices=["large", "l96_8", "l96_8_fp64", "windkessel", "windkessel_mixed",
                             "serving", "batched",
                             "precision", "variants", "samplers"])
    ap.add_argument("--cluster-bound", type=int, default=0,
                    help="batched: largest filter (particles) run on one thread-block cluster")
    ap.add_argument("--branches", type=int, default=0,
                    help="batched: independent launch chains (0: the autotuner picks the shape)")
    ap.add_argument("--rs-grid", type=int, default=4,
                    help="batched: resample blocks per SM (with --branches)")
    ap.add_argument("--persistent", type=int, default=0,
                    help="batched: CTAs per SM of the persistent launch (0: launch chains)")
    ap.add_argument("--tiles-per-item", type=int, default=1,
                    help="batched: tiles per work item of the persistent launch (1, 2, 4, 8)")
    ap.add_argument("--rates", default="250,500,1000,1500,2000", help="serving: offered rates")
    ap.add_argument("--duration", type=float, default=10.0, help="serving: seconds of arrivals")
    ap.add_argument("--drain", type=float, default=20.0, help="serving: extra seconds to finish")
    ap.add_argument("--slots", type=int, default=128, help="serving: concurrent filters")
    ap.add_argument("--server-branches", type=int, default=SERVER_BRANCHES,
                    help="serving: concurrent launch groups per scheduler iteration")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="serving: device memory budget")
    ap.add_argument("--plain-sample", type=int, default=60, help="serving: plain-form sample")
    ap.add_argument("--seeds", type=int, default=64, help="precision: seeds per configuration")
    ap.add_argument("--P", type=int, default=0, help="override the particle count")
    ap.add_argument("--T", type=int, default=0, help="override the observation count")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-peak", action="store_true")
    args = ap.parse_args()

    if args.impl == "reference":
        return run_reference(args)
    if args.config == "serving":
        return run_serving(args)
    if args.config == "precision":
        return run_precision(args)
    if args.config == "variants":
        return run_variants(args)
    if args.config == "samplers":
        return run_samplers(args)
    if args.config == "batched":
        return run_batched(args)
    args.warmup = max(args.warmup, 3)

    import torch
    import paper_1306_3277_b300 as pf

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w = make_workload(args)
    f = pf.pf_create(pf.model_from_workload(w), w.P, w.T, w.dt)
    th = torch.tensor(w.theta, dtype=torch.float64, device=dev)
    y = torch.tensor(w.y, dtype=torch.float64, device=dev)
    ll = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)
    seed0 = 1000 * (rank + 1)

    # warm-up: graph replays (the last one is timed and reported as graph_ms_per_step)
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    for k in range(args.warmup):
        if k == args.warmup - 1:
            g0.record(stream)
        pf.pf_run(f, th, y, seed0 + k, ll, None, None, pf.PF_FLAG_ASYNC, stream)
    g1.record(stream)
    stream.synchronize()
    graph_ms = g0.elapsed_time(g1)

    # timed region: K whole runs, kernels launched one by one with CUDA events
    pf.pf_profile_enable(f, True)
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        pf.pf_run(f, th, y, seed0 + 100 + k, ll, None, None, pf.PF_FLAG_ASYNC, stream)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = e0.elapsed_time(e1)
    prof = pf.pf_profile_read(f)
    pf.pf_profile_enable(f, False)
    status = pf.pf_wait(f)
    loglik = ll.item()
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)

    psteps_rank = w.P * w.T * args.steps
    value = whole_job_rate(psteps_rank, world, elapsed_ms * 1e-3)
    launches = sum(n for _, n in prof.values())

    # e2e: the public call with host buffers (H2D of theta and y, D2H of the result)
    th_h = np.ascontiguousarray(w.theta, dtype=np.float64)
    y_h = np.ascontiguousarray(w.y, dtype=np.float64)
    f.run(th_h, y_h, seed0)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        f.run(th_h, y_h, seed0 + 200 + k)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = whole_job_rate(psteps_rank, world, e2e_s)

    if rank == 0:
        peaks, peak_src = measured_peaks()
        prop_ms, prop_n = prof["propagate"]
        res_ms, res_n = prof["resample"]
        avg_prop_ms = prop_ms / max(prop_n, 1)
        avg_res_ms = res_ms / max(res_n, 1)
        if w.kind == W.LORENZ96:
            flop_launch = l96_flops_per_particle_step(w) * w.P
        else:
            flop_launch = 6 * w.substeps * w.P
        prop_bytes = propagate_bytes_per_particle(w) * w.P
        res_bytes = RESAMPLE_BYTES_PER_PARTICLE * w.P
        tag = "k_propagate<%s,%d,%s>" % ("L96" if w.kind else "WK", w.N,
                                          "f32" if w.prec else "f64")
        if prop_n == args.steps:  # a small filter: one cluster launch runs the whole run
            tag = "k_filter_cluster" + tag[len("k_propagate"):]
            flop_launch *= w.T
            prop_bytes *= w.T
        fp32_peak = fp64_peak = None
        if not args.no_peak:
            fp32_peak = pf.pf_measure_fma_peak(pf.PF_MIXED)
            fp64_peak = pf.pf_measure_fma_peak(pf.PF_FP64)
        achieved_tf = flop_launch / (avg_prop_ms * 1e-3) / 1e12
        alu_peak = fp32_peak if w.prec == W.MIXED else fp64_peak
        alu_peak_tf = alu_peak / 1e12 if alu_peak else None
        res_gbs = res_bytes / (avg_res_ms * 1e-3) / 1e9 if avg_res_ms > 0 else None
        roof = {"kernel": tag + " (fused gather, %s substeps, noise, FP64 weight, tile prefix "
                                "sums%s)" % ("RK4" if w.kind == W.LORENZ96 else "Euler",
                                             "; whole run per launch" if prop_n == args.steps
                                             else ""),
                "bound": "alu", "achieved": achieved_tf, "peak": alu_peak_tf, "unit": "TFLOP/s",
                "frac": (achieved_tf / alu_peak_tf) if alu_peak_tf else None,
                "traffic": read_traffic(tag, w.P),
                "peak_source": "measured %s FMA throughput of this GPU in this run "
                               "(pf_measure_fma_peak)" % ("FP32" if w.prec else "FP64"),
                "algorithmic_flop_per_launch": flop_launch,
                "algorithmic_bytes_per_launch": prop_bytes,
                "avg_launch_ms": avg_prop_ms, "launches": prop_n,
                "share_of_timed_region": prop_ms / elapsed_ms,
                "hbm_achieved_gbs": prop_bytes / (avg_prop_ms * 1e-3) / 1e9,
                "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peak_src,
                "fp32_fma_peak_tflops": fp32_peak / 1e12 if fp32_peak else None,
                "fp64_fma_peak_tflops": fp64_peak / 1e12 if fp64_peak else None,
                "resample_kernel": {
                    "avg_launch_ms": avg_res_ms, "launches": res_n,
                    "share_of_timed_region": res_ms / elapsed_ms,
                    "algorithmic_bytes_per_launch": res_bytes, "hbm_achieved_gbs": res_gbs,
                    "hbm_frac": res_gbs / peaks["hbm_gbs"] if res_gbs else None,
                    "traffic": read_traffic("k_resample", w.P)}}
        cpu = None
        if not args.no_cpu_baseline:
            P_s, T_s = oracle_sample(w)
            cpu_oracle_rate(w, max(P_s // 16, 1), 1)  # warm-up: library, threads, pages
            rate, secs, runs = cpu_oracle_rate(w, P_s, T_s, min_secs=5.0)
            cpu = {"value": rate, "unit": "particle-steps/s", "cores": cores(), "kind": "oracle",
                   "sample": "P=%d T=%d of the same workload, %d run(s) with seeds 1..%d, "
                             "OpenMP over particles, %.1f s wall" % (P_s, T_s, runs, runs, secs)}
        sec = None
        if not args.no_secondary and world == 1:
            sec = secondary(pf, torch, dev)
        out = {
            "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_name(w),
            "data": "synthetic (observations simulated from the model, seeded)",
            "config": {"workload": w.name, "model": "lorenz96" if w.kind else "windkessel",
                       "N": w.N, "P": w.P, "T": w.T, "substeps": w.substeps, "dt": w.dt,
                       "obs_stride": w.obs_stride, "resampling": "systematic, every step",
                       "parallelism": "%d independent replicas" % world if world > 1
                       else "single GPU",
                       "l2": l2_note(w),
                       "launch": "timed region: kernels launched one by one with per-kernel "
                                 "CUDA events; warm-up: one CUDA graph per run"},
            "graph_ms_per_step": graph_ms,
            "loglik_last": loglik, "status": pf.STATUS_NAMES[status],
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": int(y_h.nbytes + DESCRIPTOR_BYTES),
                    "d2h_bytes_per_step": 3 * 8},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "kernel_source_hash": kernel_source_hash(),
            "secondary": sec,
        }
        print(json.dumps(out), flush=True)
    f.destroy()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
