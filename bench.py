#!/usr/bin/env python
"""Benchmark of the Fchi2 periodogram hot path on one GB300 per rank.

Workload (the long single-curve case): n = 100,000 samples over 3000 d with a
seasonal window and nightly cadence, an 8-harmonic sawtooth signal, H = 6,
N = 2^22 trial frequencies up to 20 /d, grids oversampled 4x.  Inputs are
seeded synthetic curves (seed 2 + rank); every grid is larger than L2.

One step = fc2_execute on resident inputs: phase reduction, spreading, FFTs,
assembly and bordered Cholesky for all H' = 1..H, exact fix-up of sensitive
bins, peaks and coefficients.  The metric counts one evaluation per
(trial frequency, H').

--impl reference times the CPU oracle (direct sums + Householder least
squares per bin) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Delta-chi2 evals/s (freq x H') at 1e-4*chi2_0, mixed vs FP64; % HBM peak"
UNIT = "evals/s"
WORKLOAD = "long single curve: n=100000, T=3000 d seasonal+nightly, sawtooth 8 harmonics, " \
           "H=6, N=2^22 to 20/d, 4x oversampled grids"


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(ws, v):
    """Max over ranks; NCCL needs the value on this rank's GPU, gloo on the host."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        device = torch.device("cuda", torch.cuda.current_device())
    else:
        device = None
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 20 ms, started before the
    warm-up; only the samples stamped inside the timed region count."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.t0 = self.t1 = None

    def start(self):
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def begin(self):
        import datetime
        self.t0 = datetime.datetime.now()

    def end(self):
        import datetime
        self.t1 = datetime.datetime.now()

    def stop(self):
        import datetime
        if self.p is None:
            return None
        time.sleep(0.1)  # let the sampler write past the end of the region
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for ln in fh:
                parts = [x.strip() for x in ln.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                except ValueError:
                    ts = None  # unknown stamp format: the sample counts as inside
                rows.append((ts, parts[1:]))
        os.unlink(self.f.name)
        if not rows:
            return None
        pad = datetime.timedelta(milliseconds=20)
        inside = [r for ts, r in rows if ts is None or (self.t0 and self.t1 and
                                                        self.t0 - pad <= ts <= self.t1 + pad)]
        stamped = [(ts, r) for ts, r in rows if ts is not None]
        if not inside and self.t0 and stamped:  # region shorter than a sample: the nearest one
            mid = self.t0 + (self.t1 - self.t0) / 2
            inside = [min(stamped, key=lambda tr: abs(tr[0] - mid))[1]]
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(inside)}


def oracle_sample(c, bins, threads):
    from oracle import oracle
    t0 = time.perf_counter()
    d, piv = oracle.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins, threads=threads,
                               with_pivots=True)
    return d, piv, time.perf_counter() - t0


def sample_bins_for(c, n_random, seed, extra=()):
    from tests.parity import sample_bins
    f0 = c.truth.get("f0", 1.0)
    cen = [int(round((f0 - c.f_min) / c.df)), int(round((2 * f0 - c.f_min) / c.df)),
           int(round((f0 / 2 - c.f_min) / c.df)), int(round((1.0 - c.f_min) / c.df))]
    cen += [int(j) for j in extra]
    return sample_bins(c.N, n_random, seed, windows=cen, half=8)


def run_reference(args):
    ws, rank, local = dist_init()
    if rank != 0:
        return
    from paper_0901_1913_gb300 import synth
    c = synth.long_curve(seed=2)
    threads = os.cpu_count() or 1
    per_step = max(threads, args.ref_bins)
    rng = np.random.default_rng(7)
    times = []
    for it in range(args.warmup + args.steps):
        bins = np.sort(rng.choice(c.N, size=per_step, replace=False))
        _, _, dt = oracle_sample(c, bins, threads)
        if it >= args.warmup:
            times.append(dt)
    ms = 1e3 * sum(times) / len(times)
    value = per_step * c.H / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} random trial frequencies x H'=1..6 per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args):
    ws, rank, local = dist_init()
    import torch
    from paper_0901_1913_gb300 import _fc2, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    c = synth.long_curve(seed=2 + rank)
    stream = torch.cuda.Stream(device=dev)
    evals = c.N * c.H

    def make_plan(prec, t=c.t, x=c.x, s=c.sigma):
        return _fc2.Plan(t, x, s, c.H, c.f_min, c.df, c.N, c.oversample, prec,
                         stream=stream.cuda_stream, device=local, fft_kernel=args.fft_kernel,
                         fft_group=args.fft_group)

    out = torch.empty((c.H, c.N), dtype=torch.float64, device=dev)

    def timed(plan, steps, warmup, sampler=None):
        if sampler:
            sampler.start()
            time.sleep(0.3)  # the sampler is running before the timed region starts
        for _ in range(warmup):
            plan.execute(out, want_records=True)
        barrier(ws)
        torch.cuda.synchronize()
        plan.stage_timing(True)
        if sampler:
            sampler.begin()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            plan.execute(out, want_records=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.end()
        clocks = sampler.stop() if sampler else None
        barrier(ws)
        ms = e0.elapsed_time(e1)
        stage_ms, nl, fft_bytes = plan.stage_times()
        plan.stage_timing(False)
        return ms, stage_ms, nl, fft_bytes, clocks

    # --- mixed (headline) ---
    pm = make_plan("mixed")
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ms, stage_ms, nlaunch, fft_bytes, clocks = timed(pm, args.steps, args.warmup, sampler)
    counts = pm.counts
    ms_max = allreduce_max(ws, ms)
    ms_step = ms_max / args.steps
    value = ws * evals / (ms_step / 1e3)
    dm = out.cpu().numpy()
    _, best, peaks, chi0 = pm.execute(out)
    pm.close()

    # --- FP64 plain path, same workload ---
    pf = make_plan("fp64")
    f_steps = max(2, min(args.steps, args.fp64_steps))
    ms64, stage64, _, fft_bytes64, _ = timed(pf, f_steps, max(1, min(args.warmup, 2)))
    ms64_max = allreduce_max(ws, ms64)
    d64 = out.cpu().numpy()
    pf.close()
    value64 = ws * evals / (ms64_max / f_steps / 1e3)

    # --- end to end through the C ABI with host buffers ---
    tp = torch.from_numpy(np.ascontiguousarray(c.t)).pin_memory()
    xp = torch.from_numpy(np.ascontiguousarray(c.x)).pin_memory()
    sp = torch.from_numpy(np.ascontiguousarray(c.sigma)).pin_memory()
    hout = torch.empty((c.H, c.N), dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, args.e2e_steps))
    for it in range(1 + e2e_steps):
        if it == 1:
            torch.cuda.synchronize()
            barrier(ws)
            t_e2e = time.perf_counter()
        p = _fc2.Plan(tp, xp, sp, c.H, c.f_min, c.df, c.N, c.oversample, "mixed",
                      stream=stream.cuda_stream, device=local, fft_kernel=args.fft_kernel,
                      fft_group=args.fft_group)
        p.execute(hout, want_records=True)
        p.close()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t_e2e) / e2e_steps
    e2e_s = allreduce_max(ws, e2e_s)
    rec_bytes = (c.H + 8) * _fc2.ctypes.sizeof(_fc2.Best) + 8
    e2e = {"value": ws * evals / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(3 * c.n * 8), "d2h_bytes_per_step": int(c.H * c.N * 8 + rec_bytes),
           "ms_per_step": e2e_s * 1e3, "includes": "plan create (H2D, moments, tables) + execute + D2H + destroy"}

    if rank != 0:
        return

    # --- roofline of the dominant kernel (the FFT passes) ---
    peak, peak_kind = load_peaks()
    P = 2  # passes of the 2^24-point transforms at this size
    fft_ms = stage_ms[1]
    achieved = (fft_bytes / 1e9) / (fft_ms / 1e3) if fft_ms > 0 else 0.0
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "fft_pass_long_curve_traffic.txt")
    try:
        import importlib
        ver = importlib.import_module("paper_0901_1913_gb300.build").kernel_version()
        with open(tpath) as fh:
            kv = dict(ln.strip().split("=", 1) for ln in fh if "=" in ln)
        if kv.get("kernel_version") == ver and args.fft_kernel in ("default", "r64"):
            traffic = float(kv["traffic_bytes_per_launch"])
    except Exception:
        traffic = None
    kname = {"default": "k_fft_pass64", "r64": "k_fft_pass64", "r16": "k_fft_pass",
             "bulk": "k_fft_pass_tma"}[args.fft_kernel]
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": f"{kname} (2 passes/step)",
            "algorithmic_bytes_per_launch": fft_bytes / P, "launch_ms": fft_ms / P,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}

    # --- CPU oracle on a bounded sample of the same curve: baseline + parity ---
    cpu = None
    parity = None
    if not args.no_cpu and ws == 1:
        threads = os.cpu_count() or 1
        bj = [b["j"] for b in best] + [p["j"] for p in peaks if p["j"] >= 0]
        probe = sample_bins_for(c, threads, 11)[:threads]
        _, _, dt = oracle_sample(c, probe, threads)
        per_bin = dt / len(probe) * threads
        nbins = int(max(threads, min(20000, args.cpu_seconds * threads / max(per_bin, 1e-6))))
        bins = sample_bins_for(c, max(0, nbins - 9 * 17), 13, extra=bj)
        d_or, piv, dt = oracle_sample(c, bins, threads)
        cpu = {"value": len(bins) * c.H / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{len(bins)} trial frequencies x H'=1..{c.H} (random + windows at f0, "
                         f"2f0, f0/2, 1/d and the GPU's best bins)", "seconds": dt}
        from tests.parity import argmax_ok, compare
        rm = compare(dm[:, bins].T, d_or, piv, chi0)
        r6 = compare(d64[:, bins].T, d_or, piv, chi0)
        jo = int(bins[np.argmax(d_or[:, -1])])
        parity = {"bins": len(bins), "mixed_max_err_rel": rm["max_err_rel"],
                  "fp64_max_err_rel": r6["max_err_rel"], "near_alias_bins": rm["n_near_alias"],
                  "ok": bool(rm["ok"] and r6["ok"]),
                  "argmax_ok": bool(argmax_ok(best[-1]["j"], jo, d_or[:, -1], chi0, bins))}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "mixed", "n": c.n, "N": c.N, "H": c.H,
                   "oversample": c.oversample, "parallelism": f"{ws} independent curves",
                   "l2": "inputs larger than L2 (18 grids x 128 MiB)",
                   "fft_kernel": args.fft_kernel, "fft_group": args.fft_group},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(nlaunch * args.steps),
        "clocks": clocks,
        "fp64": {"value": value64, "ms_per_step": ms64_max / f_steps, "steps": f_steps,
                 "stage_ms": [round(v, 4) for v in stage64]},
        "mixed_over_fp64": value / value64,
        "stage_ms": {k: round(v, 4) for k, v in zip(["spread", "fft", "assemble", "fixup", "peaks"],
                                                    stage_ms)},
        "bins_resolved_double": counts[0], "bins_exact_sums": counts[1],
        "bins_exact_double_float": counts[2], "bins_exact_double": counts[3],
        "bins_routed_tiers": list(counts[4:7]),
        "parity": parity,
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Only `warmup + steps` mixed executes of the workload, optionally with
    fewer harmonics (--H): the command profiled by ncu.  Prints one short line
    that is not a benchmark result."""
    import torch
    from paper_0901_1913_gb300 import _fc2, synth
    if args.workload in ("survey", "adjoint"):
        b = synth.survey_batch(C=args.curves) if args.workload == "survey" else synth.adjoint_batch(C=args.curves)
        for _ in range(args.warmup + args.steps):
            _, _, stats = _fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df,
                                               b.N, b.oversample, "mixed", top_k=8,
                                               fft_kernel=args.fft_kernel)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "workload": args.workload, "curves": b.C,
                          "stats": stats}), flush=True)
        return
    c = synth.long_curve(seed=2, H=args.H or 6)
    dev = torch.device("cuda", 0)
    out = torch.empty((c.H, c.N), dtype=torch.float64, device=dev)
    with _fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed",
                   fft_kernel=args.fft_kernel, fft_group=args.fft_group) as p:
        for _ in range(args.warmup + args.steps):
            _, best, _, _ = p.execute(out, want_records=True)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "H": c.H, "N": c.N, "n": c.n,
                          "best_j": int(best[-1]["j"]), "counts": list(p.counts)}), flush=True)


WORKLOADS = {
    "short": "short single curve: n=1000 over 100 d with two gaps, 3 harmonics of 1.37/d, H=3, "
             "N=16384 on [0.01, 10]/d",
    "survey": "batched survey: 4096 curves, n ~ lognormal(median 2000) in [50, 20000], H in 2..6, "
              "N=2^18 to 12/d, 30% nulls",
    "adjoint": "differentiation batch: 1024 curves, n=2000, H=4, N=2^16 to 12/d; gradients and "
               "Newton refinement at the top-8 peaks",
    "large": "large single curve: n~1e6 at 2-min cadence over 4 yr, H=8, N=2^26 to 24/d, "
             "2x oversampled grids",
    "shared": "many sources in one field: 4096 curves sharing 2000 epochs over 1000 d, errors "
              "proportional to one set, H=4, N=2^18 to 12/d; the weights' transforms computed "
              "once per chunk",
    "paper": "long single curve (n=100000, H=6, N=2^22 to 20/d) under the paper's own gridding: "
             "nearest-lower-cell binning into one array of 2^27 cells, one transform, harmonics "
             "read at multiples of the bin index",
}


def _events_ms(fn, steps, warmup, stream=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_paper_gridding(args, line, threads):
    """The paper's own method (fc2_options.gridding = 1) on the long curve: GPU
    rates with the stage split, the same method on the host (numpy FFT and
    batched regression; the FFT in full, the regression on a sample of bins and
    scaled), parity against the oracle at the snapped times and the gridding
    error against the exact periodogram."""
    import torch
    from paper_0901_1913_gb300 import _fc2, synth
    from tests.parity import compare, sample_bins
    from oracle import oracle, paper_method
    c = synth.long_curve()
    evals = c.N * c.H
    res = {}
    for prec in ("mixed", "fp64"):
        out = torch.empty((c.H, c.N), dtype=torch.float64, device="cuda")
        with _fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec,
                       gridding="paper", fft_kernel=args.fft_kernel) as p:
            steps = args.steps if prec == "mixed" else max(2, min(args.steps, 3))
            for _ in range(max(1, min(args.warmup, 3))):
                p.execute(out, want_records=True)
            torch.cuda.synchronize()
            p.stage_timing(True)
            ms = _events_ms(lambda: p.execute(out, want_records=True), steps, 0)
            stage, _, _ = p.stage_times()
            p.stage_timing(False)
            _, best, _, chi0 = p.execute(out)
            res[prec] = (ms, out.cpu().numpy(), best, chi0, [float(v) for v in stage], p.t0)
    s0 = int(round(c.f_min / c.df))
    M = 1024
    while M < 4 * c.H * (s0 + c.N - 1) + 1:
        M *= 2
    T0 = res["fp64"][5]
    f0 = c.truth["f0"]
    bins = sample_bins(c.N, 40, 7, windows=[int(round((f0 - c.f_min) / c.df)),
                                            int(res["fp64"][2][-1]["j"])], half=2)
    tp, _ = oracle.paper_grid_times(c.t, T0, c.df, M)
    ref, piv = oracle.dchi2_bins(tp, c.x, c.sigma, c.H, c.f_min, c.df, bins, threads=threads,
                                 with_pivots=True)
    exact = oracle.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins, threads=threads)
    chi0 = res["fp64"][3]
    par = {prec: compare(res[prec][1][:, bins].T, ref, piv, chi0) for prec in res}
    # the same method on the host: full transform, regression on a sample of bins
    sample = np.unique(np.concatenate([np.arange(0, c.N, max(1, c.N // 65536)), bins]))
    d_cpu, tcpu = paper_method.fchi2_paper(c.t, c.x, c.sigma, c.H, c.f_min, c.df, sample, M, T0=T0)
    solve_full = tcpu["solve_s"] * c.N / sample.size
    cpu_total = tcpu["grid_s"] + tcpu["fft_s"] + solve_full
    idx = np.searchsorted(sample, bins)
    names = ["binning", "transform", "regression", "exact fix-up", "peaks"]
    line.update(value=evals / (res["mixed"][0] / 1e3), ms_per_step=res["mixed"][0],
                dtype="f32+f64 (mixed)",
                fp64={"value": evals / (res["fp64"][0] / 1e3), "ms_per_step": res["fp64"][0]},
                stage_ms={prec: dict(zip(names, res[prec][4])) for prec in res},
                parity_snapped_times={prec: {"max_err_rel": par[prec]["max_err_rel"],
                                              "near_alias_bins": par[prec]["n_near_alias"],
                                              "ok": bool(par[prec]["ok"])} for prec in res},
                gridding_error_vs_exact=float(np.max(np.abs(res["fp64"][1][:, bins].T - exact)) / chi0),
                cpu_baseline={"value": evals / cpu_total, "unit": UNIT, "cores": 1,
                              "kind": "paper-method (numpy FFT + batched regression, host)",
                              "sample": f"transform in full (M = {M}); regression on "
                                        f"{sample.size} of {c.N} bins, scaled",
                              "split_s": {"binning": tcpu["grid_s"], "transform": tcpu["fft_s"],
                                          "regression": solve_full},
                              "max_diff_vs_gpu_fp64_rel": float(
                                  np.max(np.abs(d_cpu[idx] - res["fp64"][1][:, bins].T)) / chi0)})
    line["config"].update(n=c.n, N=c.N, H=c.H, M=M, gridding="paper")
    print(json.dumps(line), flush=True)


def _shared_vs_independent(b, a, r):
    """Entries where the shared and independent runs differ by more than
    1e-4 chi2_0 of their curve, and the highest bin among them (they are the
    nearly singular bins at periods longer than the span)."""
    offs = np.concatenate([[0], np.cumsum(b.H.astype(np.int64) * b.N)])
    big, top_j, worst = 0, -1, 0.0
    for c in range(b.C):
        sl = slice(offs[c], offs[c + 1])
        w = 1.0 / b.sigma[b.offsets[c]:b.offsets[c + 1]] ** 2
        x = b.x[b.offsets[c]:b.offsets[c + 1]]
        xb = np.sum(w * x) / np.sum(w)
        chi0 = np.sum(w * (x - xb) ** 2)
        d = (np.abs(a[sl] - r[sl]) / chi0).reshape(int(b.H[c]), int(b.N[c]))
        worst = max(worst, float(d.max()))
        hit = np.nonzero((d > 1e-4).any(axis=0))[0]
        big += int((d > 1e-4).sum())
        if hit.size:
            top_j = max(top_j, int(hit.max()))
    return {"max_rel_chi2_0": worst, "entries_above_1e-4": big,
            "entries": int(offs[-1]), "highest_bin_above_1e-4": top_j}


def run_shared_field(args, line, threads):
    """Shared sampling (fc2_options.shared_sampling): the same batch run with
    the weights' transforms shared and as independent curves; oracle parity on
    a few curves."""
    import torch
    from paper_0901_1913_gb300 import _fc2, synth
    from tests.parity import compare, sample_bins
    from oracle import oracle
    b = synth.shared_field(C=4096)
    evals = int(np.sum(b.H.astype(np.int64) * b.N))
    dev = torch.device("cuda", 0)
    td, xd, sd = (torch.from_numpy(v).to(dev) for v in (b.t, b.x, b.sigma))
    out = torch.empty(evals, dtype=torch.float32, device=dev)
    holder = {}
    res = {}
    for shared in (True, False):
        def run():
            holder["r"] = _fc2.execute_batched(b.offsets, td, xd, sd, b.H, b.f_min, b.df, b.N,
                                               b.oversample, "mixed", top_k=8, dchi2=out,
                                               shared_sampling=shared, fft_kernel=args.fft_kernel)
        ms = _events_ms(run, args.steps, max(1, min(args.warmup, 2)))
        res[shared] = (ms, holder["r"][2], out.cpu().numpy())
    got = res[True][2]
    errs, nb = [], 0
    t0 = time.perf_counter()
    offs = np.concatenate([[0], np.cumsum(b.H.astype(np.int64) * b.N)])
    for c in range(0, b.C, 512):
        cur = b.curve(c)
        blk = got[offs[c]:offs[c + 1]].reshape(cur.H, cur.N)
        bins = sample_bins(cur.N, 24, c, windows=[0], half=2)
        ref, piv = oracle.dchi2_bins(cur.t, cur.x, cur.sigma, cur.H, cur.f_min, cur.df, bins,
                                     threads=threads, with_pivots=True)
        _, _, chi0, _ = oracle.moments(cur.x, cur.sigma)
        errs.append(compare(blk[:, bins].T.astype(np.float64), ref, piv, chi0))
        nb += len(bins) * cur.H
    dt = time.perf_counter() - t0
    line.update(value=evals / (res[True][0] / 1e3), ms_per_step=res[True][0],
                dtype="f32+f64 (mixed)", batch_stats=res[True][1],
                independent_curves={"value": evals / (res[False][0] / 1e3),
                                    "ms_per_step": res[False][0]},
                shared_over_independent=res[False][0] / res[True][0],
                vs_independent=_shared_vs_independent(b, res[True][2], res[False][2]),
                parity={"curves": len(errs), "max_err_rel": max(r["max_err_rel"] for r in errs),
                        "ok": all(r["ok"] for r in errs)},
                cpu_baseline={"value": nb / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
                              "sample": f"{nb} evals on {len(errs)} curves"},
                config=dict(line["config"], curves=b.C, samples=int(b.offsets[-1])))
    print(json.dumps(line), flush=True)


def run_workload(args):
    """The other synthetic workloads, one JSON line each (for the measurement
    table; the default run is the long curve).  Oracle parity on a bounded
    sample of bins or curves."""
    import torch
    from paper_0901_1913_gb300 import _fc2, synth
    from tests.parity import TOL, compare, sample_bins
    threads = os.cpu_count() or 1
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]}}
    if args.workload == "paper":
        run_paper_gridding(args, line, threads)
        return
    if args.workload == "shared":
        run_shared_field(args, line, threads)
        return
    if args.workload in ("short", "large"):
        c = synth.short_curve() if args.workload == "short" else synth.large_curve()
        evals = c.N * c.H
        res = {}
        for prec in ("mixed", "fp64"):
            out = torch.empty((c.H, c.N), dtype=torch.float64, device="cuda")
            with _fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec,
                           fft_kernel=args.fft_kernel) as p:
                steps = args.steps if prec == "mixed" or args.workload == "short" else 2
                ms = _events_ms(lambda: p.execute(out, want_records=True), steps,
                                max(1, min(args.warmup, 2)))
                _, best, _, chi0 = p.execute(out)
                res[prec] = (ms, out.cpu().numpy(), best, chi0, p.counts)
        if args.workload == "short":
            bins = np.arange(c.N)
        else:
            f0s = [f * h for f in c.truth["fs"] for h in (1, 2)]
            bins = sample_bins(c.N, 48, 5, windows=[int(round((f - c.f_min) / c.df))
                                                    for f in f0s] + [res["mixed"][2][-1]["j"]],
                               half=2)
        from oracle import oracle
        t0 = time.perf_counter()
        d_or, piv = oracle.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                      threads=threads, with_pivots=True)
        dt = time.perf_counter() - t0
        chi0 = res["mixed"][3]
        rm = compare(res["mixed"][1][:, bins].T, d_or, piv, chi0)
        r6 = compare(res["fp64"][1][:, bins].T, d_or, piv, chi0)
        line.update(value=evals / (res["mixed"][0] / 1e3), ms_per_step=res["mixed"][0],
                    dtype="f32+f64 (mixed)",
                    fp64={"value": evals / (res["fp64"][0] / 1e3), "ms_per_step": res["fp64"][0]},
                    mixed_over_fp64=res["fp64"][0] / res["mixed"][0],
                    counts_mixed=list(res["mixed"][4]),
                    cpu_baseline={"value": len(bins) * c.H / dt, "unit": UNIT, "cores": threads,
                                  "kind": "oracle", "sample": f"{len(bins)} bins"},
                    parity={"bins": len(bins), "mixed_max_err_rel": rm["max_err_rel"],
                            "fp64_max_err_rel": r6["max_err_rel"],
                            "near_alias_bins": rm["n_near_alias"], "ok": bool(rm["ok"] and r6["ok"])})
        line["config"].update(n=c.n, N=c.N, H=c.H, oversample=c.oversample)
    else:
        b = synth.survey_batch() if args.workload == "survey" else synth.adjoint_batch()
        evals = int(np.sum(b.H.astype(np.int64) * b.N))
        dev = torch.device("cuda", 0)
        td, xd, sd = (torch.from_numpy(v).to(dev) for v in (b.t, b.x, b.sigma))
        out = torch.empty(evals, dtype=torch.float32, device=dev)
        holder = {}

        def run(prec="mixed"):
            holder["r"] = _fc2.execute_batched(b.offsets, td, xd, sd, b.H, b.f_min, b.df, b.N,
                                               b.oversample, prec, top_k=8, dchi2=out,
                                               fft_kernel=args.fft_kernel)
        ms = _events_ms(run, args.steps, max(1, min(args.warmup, 2)))
        _, peaks, stats = holder["r"]
        got = out.cpu().numpy()
        line.update(value=evals / (ms / 1e3), ms_per_step=ms, dtype="f32+f64 (mixed)",
                    batch_stats=stats, config=dict(line["config"], curves=b.C,
                                                   samples=int(b.offsets[-1])))
        # FP64 on the first 256 curves (rate only)
        sub = min(256, b.C)
        o2 = b.offsets[:sub + 1]
        e64 = int(np.sum(b.H[:sub].astype(np.int64) * b.N[:sub]))
        t0c = time.perf_counter()
        _fc2.execute_batched(o2, b.t[:o2[-1]], b.x[:o2[-1]], b.sigma[:o2[-1]], b.H[:sub],
                             b.f_min[:sub], b.df[:sub], b.N[:sub], b.oversample, "fp64", top_k=8)
        line["fp64_first_256_curves"] = {"value": e64 / (time.perf_counter() - t0c),
                                         "note": "host-timed, includes transfers"}
        if args.workload == "adjoint":
            pj = np.array([[max(0, p_["j"]) for p_ in pk] for pk in peaks], dtype=np.int64)
            K = pj.shape[1]

            def back():
                holder["g"] = _fc2.backward_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min,
                                                    b.df, b.N, pj)
            msb = _events_ms(back, max(1, args.steps // 2), 1)
            line["backward"] = {"peaks": int(pj.size), "ms": msb,
                                "peaks_per_s": pj.size / (msb / 1e3),
                                "note": "host arrays in and out (gradients for every sample)"}
        # oracle parity on a few curves, sampled bins
        from oracle import oracle
        errs, nb, t_or = [], 0, 0.0
        pos = np.concatenate([[0], np.cumsum(b.H.astype(np.int64) * b.N)])
        for cidx in range(0, b.C, max(1, b.C // 8))[:8]:
            cur = b.curve(cidx)
            block = got[pos[cidx]:pos[cidx + 1]].reshape(cur.H, cur.N)
            bins = sample_bins(cur.N, 24, cidx, windows=[int(np.argmax(block[-1]))], half=2)
            t0c = time.perf_counter()
            ref, piv = oracle.dchi2_bins(cur.t, cur.x, cur.sigma, cur.H, cur.f_min, cur.df, bins,
                                         threads=threads, with_pivots=True)
            t_or += time.perf_counter() - t0c
            nb += len(bins) * cur.H
            _, _, chi0, _ = oracle.moments(cur.x, cur.sigma)
            errs.append(compare(block[:, bins].T.astype(np.float64), ref, piv, chi0))
        line["parity"] = {"curves": len(errs), "max_err_rel": max(e["max_err_rel"] for e in errs),
                          "ok": all(e["ok"] for e in errs)}
        line["cpu_baseline"] = {"value": nb / t_or, "unit": UNIT, "cores": threads,
                                "kind": "oracle", "sample": f"{nb} evals on {len(errs)} curves"}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fchi2", choices=["fchi2", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-bins", type=int, default=48)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="only run the mixed executes (for ncu); no benchmark line")
    ap.add_argument("--H", type=int, default=0, help="harmonics of the --profile run (default 6)")
    ap.add_argument("--workload", default="long", choices=["long"] + sorted(WORKLOADS),
                    help="long (default, the headline) or another synthetic workload")
    ap.add_argument("--fft-kernel", default="default", choices=["default", "r64", "r16", "bulk"],
                    help="kernel family of the float transform passes")
    ap.add_argument("--fft-group", type=int, default=0,
                    help="grids taken through all transform passes together (0 = all)")
    ap.add_argument("--curves", type=int, default=512,
                    help="curves of a --profile run of the survey or adjoint workload")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.workload != "long" and args.impl != "reference":
        run_workload(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
