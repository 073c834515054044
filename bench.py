#!/usr/bin/env python
"""Benchmark of the Fchi2 periodogram hot path on one GB300 per rank.

Headline workload (default): the batched survey -- 4096 light curves of
n ~ lognormal(median 2000) samples in [50, 20000] over 1000 d with seasonal
and nightly sampling, H in 2..6 harmonics, N = 2^18 trial frequencies up to
12 /d per curve, 30% pure-noise curves, grids oversampled 2x.  Inputs are
seeded synthetic curves; every chunk's grids (GBs) are larger than L2.

One step = fc2_execute_batched over the whole survey on device-resident
inputs: per curve the moments, phase reduction, spreading, FFTs, assembly and
bordered Cholesky for every H' = 1..H, the exact fix-up of sensitive bins,
and the top-8 peaks with coefficients.  The metric counts one evaluation per
(trial frequency, H').  Under torchrun each rank takes a contiguous range of
a survey of 4096 x (ranks) curves (balanced by n_c + H_c N_c; no collective on
the data path), so the work per GPU stays fixed.

The same line carries sub-records of the long single curve (n = 10^5,
N = 2^22, H = 6) and the large single curve (n ~ 10^6, N = 2^26, H = 8): mixed
and FP64 rates, their ratio, stage times and oracle parity on sampled bins.

--impl reference times the CPU oracle (direct sums + Householder least
squares per bin) on a bounded sample of the same survey.
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
SURVEY_BATCH = ("batched survey: 4096 curves per GPU, n ~ lognormal(median 2000) in [50, 20000], "
          "seasonal/nightly sampling over 1000 d, H in 2..6, N=2^18 to 12/d, 30% nulls, "
          "2x oversampled grids")
LONG = ("long single curve: n=100000, T=3000 d seasonal+nightly, sawtooth 8 harmonics, "
        "H=6, N=2^22 to 20/d, 4x oversampled grids")
LARGE = ("large single curve: n~1e6 at 2-min cadence over 4 yr, H=8, N=2^26 to 24/d, "
         "2x oversampled grids")
# Algorithmic bytes per evaluation (mixed precision): each trial frequency needs
# 3H float-complex spectrum values (Q at k = 1..2H, P at k = 1..H) written by the
# transforms and read by the assembly (2 x 24 B per (f, H')), and one float
# output per (f, H').
B_ALG = 52.0
B_FFT = 24.0    # the transforms' share: the kept spectra written


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
            else:
                torch.cuda.set_device(local)
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


def allgather(ws, obj):
    if ws == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * ws
    dist.all_gather_object(out, obj)
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profile_record(name):
    """key=value lines of a committed profile summary, or {} when missing or
    taken on other kernel sources than the ones built (its kernel_version)."""
    try:
        import importlib
        ver = importlib.import_module("paper_0901_1913_gb300.build").sources_version()
        with open(os.path.join(ROOT, "profiles", name)) as fh:
            kv = dict(ln.strip().split("=", 1) for ln in fh
                      if "=" in ln and not ln.startswith("#"))
        return kv if kv.get("kernel_version") == ver else {}
    except Exception:
        return {}


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


def sample_bins_for(c, n_random, seed, extra=(), half=8):
    from tests.parity import sample_bins
    f0 = c.truth.get("f0", 1.0)
    cen = [int(round((f0 - c.f_min) / c.df)), int(round((2 * f0 - c.f_min) / c.df)),
           int(round((f0 / 2 - c.f_min) / c.df)), int(round((1.0 - c.f_min) / c.df))]
    cen += [int(j) for j in extra]
    return sample_bins(c.N, n_random, seed, windows=cen, half=half)


def survey_for_rank(ws, rank):
    """This rank's curves of a survey of 4096 x ws curves: (batch slice as a
    synth.Batch-like namespace, (c_a, c_b))."""
    from types import SimpleNamespace

    from paper_0901_1913_gb300 import shard, synth
    full = synth.survey_batch(C=4096 * ws)
    cost = np.diff(full.offsets) + full.H.astype(np.float64) * full.N
    ca, cb = shard.curve_partition(cost, ws)[rank]
    off, (t, x, sg), (H, fm, df, N) = shard.curve_slice(full.offsets, (full.t, full.x, full.sigma),
                                                        (full.H, full.f_min, full.df, full.N),
                                                        (ca, cb))
    b = SimpleNamespace(offsets=off, t=np.ascontiguousarray(t), x=np.ascontiguousarray(x),
                        sigma=np.ascontiguousarray(sg), H=np.ascontiguousarray(H),
                        f_min=np.ascontiguousarray(fm), df=np.ascontiguousarray(df),
                        N=np.ascontiguousarray(N), oversample=full.oversample,
                        truth=full.truth[ca:cb], C=cb - ca)
    b.curve = lambda c: synth.Curve(b.t[off[c]:off[c + 1]], b.x[off[c]:off[c + 1]],
                                    b.sigma[off[c]:off[c + 1]], int(b.H[c]), float(b.f_min[c]),
                                    float(b.df[c]), int(b.N[c]), b.oversample, b.truth[c])
    return b, (ca, cb)


def run_reference(args):
    """The oracle as it stands, timed on the host cores on a bounded sample of
    the survey: each step evaluates ref_bins random trial frequencies (every
    H') on each of 4 curves spread over the batch."""
    ws, rank, local = dist_init()
    if rank != 0:
        return
    from paper_0901_1913_gb300 import synth
    b = synth.survey_batch()
    threads = os.cpu_count() or 1
    picks = [0, b.C // 4, b.C // 2, 3 * b.C // 4]
    rng = np.random.default_rng(7)
    times, evals = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ne = 0
        for ci in picks:
            c = b.curve(ci)
            bins = np.sort(rng.choice(c.N, size=max(1, args.ref_bins), replace=False))
            oracle_sample(c, bins, threads)
            ne += bins.size * c.H
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
            evals += ne
    ms = 1e3 * sum(times) / len(times)
    value = evals / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": SURVEY_BATCH, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{args.ref_bins} random trial frequencies x H'=1..H_c on each "
                                   f"of curves {picks} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def survey_parity(b, got_block, best_j, threads, seconds, n_curves=64, max_bins=1024):
    """The oracle on n_curves curves spread over the batch: per curve up to
    max_bins random trial frequencies plus +-8-bin windows at f0, 2 f0, f0/2,
    1 /d and the GPU's best bin of row H, sized so the whole sample takes about
    `seconds` on the host cores.  Returns (parity dict, cpu_baseline dict)."""
    from oracle import oracle
    from tests.parity import argmax_ok, compare
    idx = np.unique(np.linspace(0, b.C - 1, n_curves).astype(int))
    # oracle cost per bin ~ n_c H_c^3: probe it on one curve
    c0 = b.curve(int(idx[0]))
    probe = np.arange(0, c0.N, c0.N // (16 * threads))[:16 * threads]
    _, _, dt = oracle_sample(c0, probe, threads)
    per_unit = dt / (probe.size * c0.n * c0.H ** 3)
    units = sum(b.curve(int(c)).n * int(b.H[c]) ** 3 for c in idx)
    nb = int(max(16, min(max_bins, seconds / max(per_unit * units, 1e-12))))
    errs, near, nbins, nev, t_or, arg_ok = [], 0, 0, 0, 0.0, 0
    for c in idx:
        cur = b.curve(int(c))
        bins = sample_bins_for(cur, nb, int(c), extra=[best_j[c]])
        d_or, piv, dt = oracle_sample(cur, bins, threads)
        t_or += dt
        blk = got_block(int(c))
        _, _, chi0, _ = oracle.moments(cur.x, cur.sigma)
        r = compare(blk[:, bins].T.astype(np.float64), d_or, piv, chi0)
        errs.append(r)
        near += r["n_near_alias"]
        nbins += bins.size
        nev += bins.size * cur.H
        jo = int(bins[np.argmax(d_or[:, -1])])
        arg_ok += int(argmax_ok(int(best_j[c]), jo, d_or[:, -1], chi0, bins))
    parity = {"curves": int(idx.size), "bins": nbins, "evals": nev,
              "random_bins_per_curve": nb,
              "max_err_rel": max(e["max_err_rel"] for e in errs),
              "near_alias_entries": near,
              "argmax_ok": f"{arg_ok}/{idx.size}",
              "ok": bool(all(e["ok"] for e in errs) and arg_ok == idx.size)}
    cpu = {"value": nev / t_or, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{nbins} trial frequencies x H'=1..H_c on {idx.size} curves spread over the "
                     f"batch ({nb} random per curve + windows at f0, 2f0, f0/2, 1/d and the "
                     f"GPU's best bin)", "seconds": t_or}
    return parity, cpu


def single_curve_record(c, args, threads, n_random, half, mixed_steps, fp64_steps, windows,
                        first_bins=0):
    """Mixed and FP64 rates of one curve (CUDA events on the plan's stream),
    stage times, and oracle parity on sampled bins (random ones, windows at the
    given bins and the best one, and the first `first_bins` bins: periods
    longer than the span, the exact fix-up's hardest cases)."""
    import torch
    from paper_0901_1913_gb300 import _fc2
    from tests.parity import compare, sample_bins
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    out = torch.empty((c.H, c.N), dtype=torch.float64, device=dev)
    res = {}
    for prec, steps in (("mixed", mixed_steps), ("fp64", fp64_steps)):
        with _fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec,
                       stream=stream.cuda_stream, device=dev.index) as p:
            p.execute(out)
            torch.cuda.synchronize()
            p.stage_timing(True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                p.execute(out, want_records=True)
            e1.record(stream)
            torch.cuda.synchronize()
            stage, nl, _ = p.stage_times()
            p.stage_timing(False)
            _, best, _, chi0 = p.execute(out)
            res[prec] = dict(ms=e0.elapsed_time(e1) / steps, d=out.cpu().numpy(), best=best,
                             chi0=chi0, stage=[round(float(v), 4) for v in stage],
                             counts=list(p.counts), launches=nl)
    evals = c.N * c.H
    bins = sample_bins(c.N, n_random, 11, windows=list(windows) + [res["mixed"]["best"][-1]["j"]],
                       half=half)
    bins = np.union1d(bins, np.arange(min(first_bins, c.N), dtype=np.int64))
    from oracle import oracle
    t0 = time.perf_counter()
    d_or, piv = oracle.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins, threads=threads,
                                  with_pivots=True)
    dt = time.perf_counter() - t0
    chi0 = res["fp64"]["chi0"]
    rm = compare(res["mixed"]["d"][:, bins].T, d_or, piv, chi0)
    r6 = compare(res["fp64"]["d"][:, bins].T, d_or, piv, chi0)
    names = ["spread", "fft", "assemble", "fixup", "peaks"]
    return {
        "n": c.n, "N": c.N, "H": c.H, "oversample": c.oversample,
        "mixed": {"value": evals / (res["mixed"]["ms"] / 1e3), "ms_per_step": res["mixed"]["ms"],
                  "steps": mixed_steps, "stage_ms": dict(zip(names, res["mixed"]["stage"])),
                  "bins_resolved_double": res["mixed"]["counts"][0],
                  "bins_exact_sums": res["mixed"]["counts"][1],
                  "bins_through_tiers_2_3": res["mixed"]["counts"][2:4]},
        "fp64": {"value": evals / (res["fp64"]["ms"] / 1e3), "ms_per_step": res["fp64"]["ms"],
                 "steps": fp64_steps, "stage_ms": dict(zip(names, res["fp64"]["stage"]))},
        "mixed_over_fp64": res["fp64"]["ms"] / res["mixed"]["ms"],
        "parity": {"bins": int(bins.size), "mixed_max_err_rel": rm["max_err_rel"],
                   "fp64_max_err_rel": r6["max_err_rel"], "near_alias_bins": rm["n_near_alias"],
                   "ok": bool(rm["ok"] and r6["ok"])},
        "oracle": {"value": bins.size * c.H / dt, "unit": UNIT, "cores": threads,
                   "seconds": dt},
    }


class PinnedHost:
    """A page-locked host array of exactly n float32 elements, allocated with
    cudaHostAlloc from the CUDA runtime the library loaded (the caching pinned
    allocator of torch rounds a request up to a power of two: 32 GB for the
    survey's 17.2 GB periodogram).  .tensor is a torch CPU view; close()
    frees it."""

    def __init__(self, n):
        import ctypes
        import torch
        path = None
        with open("/proc/self/maps") as fh:
            for line in fh:
                if "libcudart.so" in line:
                    path = line.split()[-1]
                    break
        if path is None:
            raise RuntimeError("the CUDA runtime is not loaded")
        self._rt = ctypes.CDLL(path)
        self._ptr = ctypes.c_void_p()
        rc = self._rt.cudaHostAlloc(ctypes.byref(self._ptr), ctypes.c_size_t(4 * n),
                                    ctypes.c_uint(1))  # cudaHostAllocPortable: every context
        if rc != 0 or not self._ptr.value:
            raise RuntimeError(f"cudaHostAlloc of {4 * n} bytes failed ({rc})")
        buf = (ctypes.c_float * n).from_address(self._ptr.value)
        self.tensor = torch.from_numpy(np.ctypeslib.as_array(buf))

    def close(self):
        import ctypes
        if self._ptr.value:
            self.tensor = None
            self._rt.cudaFreeHost(self._ptr)
            self._ptr = ctypes.c_void_p()


def host_link_probe(hbuf, dev, stream):
    """GB/s of one 2 GB copy each way between a device buffer and the pinned
    host buffer `hbuf` (float32), timed with CUDA events: the host link's
    state when the end-to-end steps ran (the link is shared with the
    machine's other GPUs and jobs)."""
    import torch
    n = min(hbuf.numel(), 512 << 20)
    d = torch.empty(n, dtype=torch.float32, device=dev)
    out = {}
    for name in ("d2h", "h2d"):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            if name == "d2h":
                hbuf[:n].copy_(d, non_blocking=True)
            else:
                d.copy_(hbuf[:n], non_blocking=True)
            e1.record(stream)
        stream.synchronize()
        out[name] = round(4 * n / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    del d
    return out


def run_survey(args):
    ws, rank, local = dist_init()
    import torch
    from paper_0901_1913_gb300 import _fc2, synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b, (ca, cb) = survey_for_rank(ws, rank)
    evals = int(np.sum(b.H.astype(np.int64) * b.N))
    K = 8
    stream = torch.cuda.Stream(device=dev)
    pos = np.concatenate([[0], np.cumsum(b.H.astype(np.int64) * b.N)])

    def call(t, x, s, out, prec="mixed", sub=None, autotune="table"):
        off, H, fm, df, N = b.offsets, b.H, b.f_min, b.df, b.N
        if sub is not None:
            off, H, fm, df, N = off[:sub + 1], H[:sub], fm[:sub], df[:sub], N[:sub]
            t, x, s = t[:int(off[-1])], x[:int(off[-1])], s[:int(off[-1])]
        return _fc2.execute_batched(off, t, x, s, H, fm, df, N, b.oversample, prec, top_k=K,
                                    dchi2=out, stream=stream.cuda_stream, device=local,
                                    autotune=autotune)

    # ---- end to end through the C ABI with host buffers; the process's first
    # library call is the cold one (graph instantiation, pool growth, tables)
    tp, xp, sp = (torch.from_numpy(v).pin_memory() for v in (b.t, b.x, b.sigma))
    _fc2.load()
    hbuf = PinnedHost(evals)
    hout = hbuf.tensor
    barrier(ws)
    t0 = time.perf_counter()
    _, _, st_cold = call(tp, xp, sp, hout)
    cold_ms = allreduce_max(ws, (time.perf_counter() - t0) * 1e3)
    cold_cfg = st_cold["config"]
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        _, _, st_e2e = call(tp, xp, sp, hout)
    e2e_s = allreduce_max(ws, (time.perf_counter() - t0) / e2e_steps)
    link = host_link_probe(hout, dev, stream)
    del hout
    hbuf.close()

    # ---- device-resident inputs and output: the headline
    td, xd, sd = (torch.from_numpy(v).to(dev) for v in (b.t, b.x, b.sigma))
    out = torch.empty(evals, dtype=torch.float32, device=dev)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    for _ in range(args.warmup):
        call(td, xd, sd, out)
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        _, peaks, stats = call(td, xd, sd, out)
    e1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.end()
    clocks = sampler.stop() if sampler else None
    barrier(ws)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = allreduce_max(ws, ms)
    total_evals = sum(allgather(ws, evals))
    value = total_evals / (ms_max / 1e3)

    # ---- the stage split, from separate calls with stage events (each chunk is
    # then waited for, so these calls run slightly slower than the timed ones)
    _fc2.batch_timing(True)
    stage_sum = dict.fromkeys(_fc2.BATCH_STAGES, 0.0)
    fft_alg = 0.0
    n_stage = max(1, min(args.steps, 3))
    for _ in range(n_stage):
        _, _, st_stage = call(td, xd, sd, out)
        for k, v in st_stage["stage_ms"].items():
            stage_sum[k] += v
        fft_alg += st_stage["fft_alg_bytes"]
    _fc2.batch_timing(False)
    stage_ms = {k: v / n_stage for k, v in stage_sum.items()}
    fft_alg /= n_stage

    # ---- the fixed default launch configuration, against the tuned one
    call(td, xd, sd, out, autotune="fixed")
    torch.cuda.synchronize()
    x0e = torch.cuda.Event(enable_timing=True)
    x1e = torch.cuda.Event(enable_timing=True)
    x0e.record(stream)
    for _ in range(2):
        call(td, xd, sd, out, autotune="fixed")
    x1e.record(stream)
    torch.cuda.synchronize()
    ms_fixed = allreduce_max(ws, x0e.elapsed_time(x1e) / 2)

    # ---- FP64 on the first 256 curves (device-resident, CUDA events)
    sub = min(256, b.C)
    e64 = int(pos[sub])
    out64 = torch.empty(e64, dtype=torch.float32, device=dev)
    call(td, xd, sd, out64, "fp64", sub)
    torch.cuda.synchronize()
    f0e = torch.cuda.Event(enable_timing=True)
    f1e = torch.cuda.Event(enable_timing=True)
    f0e.record(stream)
    for _ in range(2):
        call(td, xd, sd, out64, "fp64", sub)
    f1e.record(stream)
    torch.cuda.synchronize()
    ms64 = allreduce_max(ws, f0e.elapsed_time(f1e) / 2)
    value64 = sum(allgather(ws, e64)) / (ms64 / 1e3)
    del out64

    # ---- the long curve split into bands over the ranks (records all-gathered)
    band = None
    if ws > 1 and not args.no_sub:
        band = run_long_bands(ws, rank, local)

    if rank != 0:
        return

    peak, peak_kind = load_peaks()
    prof = profile_record("survey_traffic.txt")
    traffic = float(prof["traffic_bytes_per_step"]) if "traffic_bytes_per_step" in prof else None
    roof = {"bound": "hbm", "achieved": value * B_ALG / 1e9, "peak": peak, "unit": "GB/s",
            "frac": value * B_ALG / 1e9 / peak, "traffic": traffic,
            "kernel": "the whole fc2_execute_batched step (every kernel of the survey pipeline)",
            "algorithmic_bytes_per_eval": B_ALG,
            "algorithmic_bytes_per_step": evals * B_ALG,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    fft_ms = stage_ms["fft"]
    cfg = stats["config"]
    dominant = {"name": "transform passes (log2 radices %s, %s)" % (
                    " x ".join(str(r) for r in cfg["fft_log2_radices"]), cfg["fft_family"]),
                "ms_per_step": fft_ms, "algorithmic_bytes_per_step": fft_alg,
                "achieved": fft_alg / 1e9 / (fft_ms / 1e3) if fft_ms > 0 else None,
                "frac": (fft_alg / 1e9 / (fft_ms / 1e3)) / peak if fft_ms > 0 else None,
                "unit": "GB/s", "traffic_bytes_per_step": (float(prof["fft_traffic_bytes_per_step"])
                                                        if "fft_traffic_bytes_per_step" in prof
                                                        else None)}
    dram_frac = float(prof["dram_frac_byte_weighted"]) if "dram_frac_byte_weighted" in prof else None

    parity = cpu = None
    if not args.no_cpu and ws == 1:
        best_j = np.array([int(pk[0]["j"]) if pk[0]["j"] >= 0 else 0
                           for pk in (peaks[c] for c in range(b.C))])

        def block(c):
            return out[int(pos[c]):int(pos[c + 1])].cpu().numpy().reshape(int(b.H[c]), int(b.N[c]))
        parity, cpu = survey_parity(b, block, best_j, os.cpu_count() or 1, args.cpu_seconds)

    subrec = {}
    if ws == 1 and not args.no_sub:
        threads = os.cpu_count() or 1
        c = synth.long_curve()
        f0 = c.truth["f0"]
        subrec["long_curve"] = dict(workload=LONG, **single_curve_record(
            c, args, threads, 1024, 8, min(args.steps, 20), 3,
            [round((k * f0 - c.f_min) / c.df) for k in (0.5, 1, 2)] + [round((1 - c.f_min) / c.df)],
            first_bins=32))
        del c
        c = synth.large_curve()
        subrec["large_curve"] = dict(workload=LARGE, **single_curve_record(
            c, args, threads, 192, 2, 3, 2,
            [round((f * h - c.f_min) / c.df) for f in c.truth["fs"] for h in (1, 2)],
            first_bins=32))
        del c
    if band is not None:
        subrec["long_curve_bands"] = band

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": SURVEY_BATCH, "curves_per_gpu": b.C, "samples": int(b.offsets[-1]),
                   "evals_per_step": evals, "N": int(b.N[0]), "H": "2..6",
                   "oversample": int(b.oversample), "precision": "mixed",
                   "parallelism": f"{ws} rank(s), contiguous curve ranges, no data-path collective",
                   "l2": "inputs larger than L2 (each chunk's grids hold several GB)"},
        "roofline": roof,
        "dominant_kernel": dominant,
        "dram_frac": dram_frac,
        "cpu_baseline": cpu,
        "e2e": {"value": total_evals / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": int(3 * 8 * int(b.offsets[-1])),
                "d2h_bytes_per_step": int(4 * evals + b.C * K * _fc2.BEST_DTYPE.itemsize),
                "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
                "host_link_gbs_after": link,
                "cold_first_call_ms": cold_ms,
                "host_phase_ms_last_call": {k: round(v, 2) for k, v in
                                            st_e2e["host_phase_ms"].items()},
                "includes": "fc2_execute_batched from pinned host arrays (t, x, sigma) to pinned "
                            "host Delta chi^2 (one exact-size cudaHostAlloc buffer) and peak "
                            "records; the cold call is the process's first library call"},
        "gpu_launches": int(stats["launches"] * args.steps),
        "clocks": clocks,
        "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()},
        "batch_stats": {k: stats[k] for k in ("resolved", "exact", "exact_double_float",
                                              "exact_double", "graphs")},
        "fp64_first_256_curves": {"value": value64, "ms_per_step": ms64,
                                  "evals_per_step": e64},
        "mixed_over_fp64_batched": value / value64,
        "autotune": {"choice": {k: v for k, v in stats["config"].items()
                                if k not in ("configurations_timed", "tuning_ms")},
                     "source_in_timed_steps": stats["config"]["source"],
                     "tuned_in_first_call": {k: cold_cfg[k] for k in
                                             ("source", "configurations_timed", "tuning_ms")},
                     "ms_per_step_tuned": ms_max, "ms_per_step_fixed_default": ms_fixed,
                     "fixed_over_tuned": ms_fixed / ms_max},
        "parity": parity,
        **subrec,
    }
    if "long_curve" in subrec:
        line["mixed_over_fp64_single_curve"] = value / subrec["long_curve"]["fp64"]["value"]
    print(json.dumps(line), flush=True)


def run_long_bands(ws, rank, local):
    """The long curve's trial range split into one band per rank (shard.run_band):
    each rank transforms and solves its own band; the per-band records are
    all-gathered and merged.  Timed by CUDA events on the plans' stream."""
    import torch
    from paper_0901_1913_gb300 import _fc2, shard, synth
    c = synth.long_curve()
    stream = torch.cuda.Stream(device=torch.device("cuda", local))

    def make_plan(fm, nb, k):
        return _fc2.Plan(c.t, c.x, c.sigma, c.H, fm, c.df, nb, c.oversample, "mixed", top_k=k,
                         stream=stream.cuda_stream, device=local)

    def gather(obj):
        return allgather(ws, obj)

    shard.run_band(make_plan, c.f_min, c.df, c.N, 8, rank, ws, gather)  # warm-up
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    band, _, best, peaks, _ = shard.run_band(make_plan, c.f_min, c.df, c.N, 8, rank, ws, gather)
    torch.cuda.synchronize()
    s = allreduce_max(ws, time.perf_counter() - t0)
    return {"workload": LONG, "bands": ws, "value": c.N * c.H / s, "ms_per_step": s * 1e3,
            "includes": "plan creation per band, execute, records all-gather and merge",
            "best_H_j": int(best[-1]["j"]), "top_peak_j": int(peaks[0]["j"]) if peaks else -1}


def run_long(args):
    """The long single curve alone (--workload long): mixed rate with stage
    times, FP64 rate, the transform's roofline, oracle parity."""
    ws, rank, local = dist_init()
    import torch
    from paper_0901_1913_gb300 import synth
    torch.cuda.set_device(local)
    c = synth.long_curve(seed=2 + rank)
    threads = os.cpu_count() or 1
    f0 = c.truth["f0"]
    rec = single_curve_record(c, args, threads, 1024, 8, args.steps, 3,
                              [round((k * f0 - c.f_min) / c.df) for k in (0.5, 1, 2)] +
                              [round((1 - c.f_min) / c.df)])
    if rank != 0:
        return
    line = {"metric": METRIC, "value": rec["mixed"]["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": rec["mixed"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)",
            "data": "synthetic", "config": {"workload": LONG}, **rec}
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Only `warmup + steps` mixed executes of the workload (the survey, the
    differentiation batch, the large curve, else the long curve, optionally with
    fewer harmonics (--H)): the command profiled by ncu.  Prints one short line
    that is not a benchmark result."""
    import torch
    from paper_0901_1913_gb300 import _fc2, synth
    if args.workload in ("survey", "adjoint"):
        b = synth.survey_batch(C=args.curves) if args.workload == "survey" else synth.adjoint_batch(C=args.curves)
        for _ in range(args.warmup + args.steps):
            _, _, stats = _fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df,
                                               b.N, b.oversample, "mixed", top_k=8,
                                               fft_kernel=args.fft_kernel,
                                               autotune=args.autotune)
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": True, "workload": args.workload, "curves": b.C,
                          "stats": stats}), flush=True)
        return
    if args.workload == "large":
        c = synth.large_curve(N=args.N) if args.N else synth.large_curve()
    else:
        c = synth.long_curve(seed=2, H=args.H or 6, **({"N": args.N} if args.N else {}))
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
    table; the default run is the survey).  Oracle parity on a bounded sample
    of bins or curves."""
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
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--autotune", default="table", choices=("table", "fixed", "retune"),
                    help="batched launch configuration in --profile runs: the tuning table "
                         "(tuning on a miss), the fixed default, or tuned anew")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--ref-bins", type=int, default=128)
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle (parity, cpu_baseline)")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the single-curve sub-records of the default run")
    ap.add_argument("--profile", action="store_true",
                    help="only run the mixed executes (for ncu); no benchmark line")
    ap.add_argument("--H", type=int, default=0, help="harmonics of the --profile run (default 6)")
    ap.add_argument("--N", type=int, default=0,
                    help="trial frequencies of a --profile run of the large curve (default 2^26)")
    ap.add_argument("--workload", default="survey", choices=["survey", "long"] + sorted(k for k in WORKLOADS if k != "survey"),
                    help="survey (default, the headline) or another synthetic workload")
    ap.add_argument("--fft-kernel", default="default", choices=["default", "r64", "r16", "bulk", "r32", "r32x"],
                    help="kernel family of the float transform passes")
    ap.add_argument("--fft-group", type=int, default=0,
                    help="grids taken through all transform passes together (0 = all)")
    ap.add_argument("--curves", type=int, default=512,
                    help="curves of a --profile run of the survey or adjoint workload")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    elif args.workload == "survey":
        run_survey(args)
    elif args.workload == "long":
        run_long(args)
    else:
        run_workload(args)


if __name__ == "__main__":
    main()
