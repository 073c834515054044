"""ctypes binding of libfc2 (the C ABI declared in include/fc2.h).

Argument marshalling only: every step of the periodogram runs in the CUDA
library.  The library is built in-tree by ``paper_0901_1913_gb300.build``; if
it is missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfc2.so")
MAX_H = 16

FC2_OK, FC2_ERR_INVALID_ARG, FC2_ERR_CUDA, FC2_ERR_OOM, FC2_ERR_TIMEOUT, \
    FC2_ERR_UNSUPPORTED, FC2_ERR_NUMERIC = range(7)
FC2_PREC_FP64, FC2_PREC_MIXED = 0, 1
PREC = {"fp64": FC2_PREC_FP64, "mixed": FC2_PREC_MIXED}


class Options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("kernel_width", ctypes.c_int), ("top_k", ctypes.c_int),
                ("alias_tau", ctypes.c_double), ("cuda_stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("inputs_on_device", ctypes.c_int),
                ("outputs_on_device", ctypes.c_int), ("autotune", ctypes.c_int),
                ("fft_kernel", ctypes.c_int), ("gridding", ctypes.c_int),
                ("detrend", ctypes.c_int), ("shared_sampling", ctypes.c_int),
                ("fft_group", ctypes.c_int), ("trend_fit", ctypes.c_int)]

# fc2_options.gridding values
GRIDDING = {"kernel": 0, "paper": 1}

# fc2_options.fft_kernel values
FFT_KERNELS = {"default": 0, "r64": 1, "r16": 2, "bulk": 3, "r32": 4, "r32x": 5}


class Best(ctypes.Structure):
    _fields_ = [("j", ctypes.c_int64), ("f", ctypes.c_double), ("dchi2", ctypes.c_double),
                ("H", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("A", ctypes.c_double * (2 * MAX_H + 1))]

    def as_dict(self):
        m = 2 * self.H + 1
        return dict(j=int(self.j), f=float(self.f), dchi2=float(self.dchi2), H=int(self.H),
                    flags=int(self.flags), A=np.array(self.A[:m]))


# the same record as a numpy structured type (fields in fc2_best order)
BEST_DTYPE = np.dtype([("j", "<i8"), ("f", "<f8"), ("dchi2", "<f8"), ("H", "<i4"),
                       ("flags", "<i4"), ("A", "<f8", (2 * MAX_H + 1,))])
assert BEST_DTYPE.itemsize == ctypes.sizeof(Best)


def _rec_dict(r):
    m = 2 * int(r["H"]) + 1
    return dict(j=int(r["j"]), f=float(r["f"]), dchi2=float(r["dchi2"]), H=int(r["H"]),
                flags=int(r["flags"]), A=np.array(r["A"][:m]))


class BatchPeaks:
    """Peak records of a batched call.  ``peaks[c]`` is curve c's list of K
    records as dicts (made when accessed; keys as ``Best.as_dict``);
    ``records`` is the structured array [C, K] of ``BEST_DTYPE``."""

    def __init__(self, records):
        self.records = records

    def __len__(self):
        return self.records.shape[0]

    def __getitem__(self, c):
        if isinstance(c, slice):
            return [self[i] for i in range(*c.indices(len(self)))]
        return [_rec_dict(r) for r in self.records[c]]

    def __iter__(self):
        for c in range(len(self)):
            yield self[c]


class Fc2Error(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def load():
    """Load libfc2.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfc2.so not built ({LIB_PATH}); run paper_0901_1913_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.fc2_options_default.argtypes = [ctypes.POINTER(Options)]
        lib.fc2_options_default.restype = None
        lib.fc2_plan_create.argtypes = [_P, _P, _P, i64, i32, dbl, dbl, i64, i32,
                                        ctypes.POINTER(Options), ctypes.POINTER(_P)]
        lib.fc2_plan_create.restype = i32
        lib.fc2_execute.argtypes = [_P, _P, _P, _P, _P]
        lib.fc2_execute.restype = i32
        lib.fc2_execute_batched.argtypes = [i64, _P, _P, _P, _P, _P, _P, _P, _P, i32,
                                            ctypes.POINTER(Options), _P, _P]
        lib.fc2_execute_batched.restype = i32
        lib.fc2_backward.argtypes = [_P, i32, _P, _P, _P, _P, _P, _P, _P]
        lib.fc2_backward.restype = i32
        lib.fc2_plan_destroy.argtypes = [_P]
        lib.fc2_plan_destroy.restype = None
        lib.fc2_status_string.argtypes = [i32]
        lib.fc2_status_string.restype = ctypes.c_char_p
        lib.fc2_grid_size.argtypes = [i64, i32]
        lib.fc2_grid_size.restype = i64
        lib.fc2_default_width.argtypes = [i32, i32]
        lib.fc2_default_width.restype = i32
        lib.fc2_kernel_ft.argtypes = [i32, i32, _P, i64, _P]
        lib.fc2_kernel_ft.restype = i32
        lib.fc2_kernel_eval.argtypes = [i32, i32, _P, i64, _P]
        lib.fc2_kernel_eval.restype = i32
        lib.fc2_debug_flag_count.argtypes = [_P]
        lib.fc2_debug_flag_count.restype = i64
        lib.fc2_debug_spectra.argtypes = [_P, _P, _P]
        lib.fc2_debug_spectra.restype = i32
        lib.fc2_debug_counts.argtypes = [_P, _P]
        lib.fc2_debug_counts.restype = None
        lib.fc2_debug_batch_launches.argtypes = []
        lib.fc2_debug_batch_launches.restype = i64
        lib.fc2_debug_batch_counts.argtypes = [_P]
        lib.fc2_debug_batch_counts.restype = None
        lib.fc2_debug_batch_phase_ms.argtypes = [_P]
        lib.fc2_debug_batch_phase_ms.restype = None
        lib.fc2_stage_timing.argtypes = [_P, i32]
        lib.fc2_stage_timing.restype = i32
        lib.fc2_stage_times.argtypes = [_P, _P, _P, _P]
        lib.fc2_stage_times.restype = i32
        lib.fc2_debug_exact_bins.argtypes = [_P, _P, i64, i32, _P]
        lib.fc2_debug_exact_bins.restype = i32
        lib.fc2_debug_tier_bins.argtypes = [_P, i32, _P, i64]
        lib.fc2_debug_tier_bins.restype = i64
        lib.fc2_trim_device_memory.argtypes = [i32]
        lib.fc2_trim_device_memory.restype = i32
        lib.fc2_debug_t0.argtypes = [_P]
        lib.fc2_debug_t0.restype = dbl
        lib.fc2_significance.argtypes = [_P, _P, _P, _P, _P]
        lib.fc2_significance.restype = i32
        lib.fc2_debug_batch_timing.argtypes = [i32]
        lib.fc2_debug_batch_timing.restype = None
        lib.fc2_debug_batch_stage_ms.argtypes = [_P]
        lib.fc2_debug_batch_stage_ms.restype = None
        lib.fc2_debug_fault.argtypes = [_P, ctypes.c_longlong, i32]
        lib.fc2_debug_fault.restype = i32
        lib.fc2_debug_last_tier.argtypes = [i32]
        lib.fc2_debug_last_tier.restype = None
        lib.fc2_debug_fail_alloc.argtypes = [i64]
        lib.fc2_debug_fail_alloc.restype = None
        lib.fc2_debug_alloc_count.argtypes = []
        lib.fc2_debug_alloc_count.restype = i64
        lib.fc2_debug_pool_used.argtypes = [i32]
        lib.fc2_debug_pool_used.restype = i64
        lib.fc2_debug_batch_config.argtypes = [_P]
        lib.fc2_debug_batch_config.restype = None
        lib.fc2_debug_batch_force.argtypes = [i32, i32, i32, i32]
        lib.fc2_debug_batch_force.restype = None
        lib.fc2_debug_batch_force_plan.argtypes = [_P, i32, i32]
        lib.fc2_debug_batch_force_plan.restype = None
        lib.fc2_debug_batch_forget_tuning.argtypes = []
        lib.fc2_debug_batch_forget_tuning.restype = None
        lib.fc2_debug_spread_force_general.argtypes = [i32]
        lib.fc2_debug_spread_force_general.restype = None
        _lib = lib
        return lib


def status_string(code):
    return load().fc2_status_string(int(code)).decode()


def _check(rc, where):
    if rc != FC2_OK:
        raise Fc2Error(rc, where)


def _ptr(a):
    """Address of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_dev(a):
    return (not isinstance(a, np.ndarray)) and getattr(a, "is_cuda", False)


def make_options(prec="fp64", kernel_width=0, top_k=0, alias_tau=0.0, stream=None, device=0,
                 inputs_on_device=False, outputs_on_device=False, autotune=False,
                 fft_kernel="default", gridding="kernel", detrend=0, shared_sampling=False,
                 fft_group=0, trend_fit=False):
    o = Options()
    load().fc2_options_default(ctypes.byref(o))
    o.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    o.kernel_width = int(kernel_width)
    o.top_k = int(top_k)
    o.alias_tau = float(alias_tau)
    o.cuda_stream = stream
    o.device = int(device)
    o.inputs_on_device = int(bool(inputs_on_device))
    o.outputs_on_device = int(bool(outputs_on_device))
    o.autotune = AUTOTUNE[autotune] if isinstance(autotune, str) else int(autotune)
    o.fft_kernel = FFT_KERNELS[fft_kernel] if isinstance(fft_kernel, str) else int(fft_kernel)
    o.gridding = GRIDDING[gridding] if isinstance(gridding, str) else int(gridding)
    o.detrend = int(detrend)
    o.shared_sampling = int(bool(shared_sampling))
    o.fft_group = int(fft_group)
    o.trend_fit = int(bool(trend_fit))
    return o


class Plan:
    """Owns an fc2_plan.  t, x, sigma: float64 numpy arrays (copied to the
    device) or float64 CUDA tensors (borrowed; keep them alive)."""

    def __init__(self, t, x, sigma, H, f_min, df, N, oversample=2, prec="fp64",
                 kernel_width=0, top_k=8, alias_tau=0.0, stream=None, device=0,
                 autotune=False, fft_kernel="default", gridding="kernel", detrend=0,
                 fft_group=0, trend_fit=False):
        lib = load()
        dev = _is_dev(t)
        if not dev:
            t = np.ascontiguousarray(t, dtype=np.float64)
            x = np.ascontiguousarray(x, dtype=np.float64)
            sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        self._keep = (t, x, sigma)
        self.n = int(t.shape[0])
        self.H, self.N, self.top_k = int(H), int(N), int(top_k or 8)
        self.f_min, self.df = float(f_min), float(df)
        self.opt = make_options(prec, kernel_width, self.top_k, alias_tau, stream, device,
                                autotune=autotune, fft_kernel=fft_kernel, gridding=gridding,
                                detrend=detrend, fft_group=fft_group, inputs_on_device=dev,
                                trend_fit=trend_fit)
        h = _P()
        rc = lib.fc2_plan_create(_ptr(t), _ptr(x), _ptr(sigma), self.n, self.H, self.f_min,
                                 self.df, self.N, int(oversample), ctypes.byref(self.opt),
                                 ctypes.byref(h))
        _check(rc, "fc2_plan_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().fc2_plan_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def execute(self, dchi2=None, want_records=True):
        """Run the periodogram.  dchi2: optional preallocated [H, N] float64
        output (numpy, or CUDA tensor when the plan writes device outputs).
        Returns (dchi2, best[H], peaks[top_k], chi2_0)."""
        lib = load()
        if dchi2 is None:
            dchi2 = np.empty((self.H, self.N), dtype=np.float64)
        best = (Best * self.H)()
        peaks = (Best * self.top_k)()
        chi0 = ctypes.c_double()
        rc = self._execute(lib, dchi2, best if want_records else None,
                           peaks if want_records else None, chi0)
        _check(rc, "fc2_execute")
        return dchi2, [b.as_dict() for b in best], [p.as_dict() for p in peaks], chi0.value

    def _execute(self, lib, dchi2, best, peaks, chi0):
        return lib.fc2_execute(self.h, _ptr(dchi2), ctypes.cast(best, _P) if best else None,
                               ctypes.cast(peaks, _P) if peaks else None, ctypes.byref(chi0))

    @property
    def flag_count(self):
        return int(load().fc2_debug_flag_count(self.h))

    @property
    def counts(self):
        """(bins re-solved in double, bins recomputed from exact sums, bins
        through double-float sums, bins through all-double sums, then the bins
        first routed to tiers 1, 2, 3) in the last execute."""
        c = np.zeros(7, dtype=np.int64)
        load().fc2_debug_counts(self.h, c.ctypes.data)
        return tuple(int(v) for v in c)

    def tier_bins(self, tier, cap=1 << 16):
        """Bins of the last execute handled by fix-up tier 2 or 3."""
        out = np.empty(cap, dtype=np.int64)
        nb = load().fc2_debug_tier_bins(self.h, int(tier), out.ctypes.data, cap)
        if nb < 0:
            raise RuntimeError("tier_bins failed")
        return out[:nb].copy()

    def exact_bins(self, bins, tier):
        """Delta chi^2 [H, len(bins)] at the given bins from the exact sums of one
        tier (1 float, 2 double-float, 3 double, 4 double-float terms with
        sums exact in fixed point)."""
        b = np.ascontiguousarray(bins, dtype=np.int64)
        out = np.empty((self.H, b.size))
        _check(load().fc2_debug_exact_bins(self.h, b.ctypes.data, b.size, int(tier),
                                           out.ctypes.data), "exact_bins")
        return out

    def spectra(self):
        G = 3 * self.H
        re = np.empty(G * self.N)
        im = np.empty(G * self.N)
        _check(load().fc2_debug_spectra(self.h, re.ctypes.data, im.ctypes.data), "spectra")
        return (re + 1j * im).reshape(G, self.N)

    def stage_timing(self, enable=True):
        _check(load().fc2_stage_timing(self.h, int(enable)), "fc2_stage_timing")

    def stage_times(self):
        """(mean ms per execute of [spread, fft, assemble, fix-up, peaks],
        kernels launched by the last execute, FFT algorithmic bytes)."""
        ms = np.zeros(5)
        nl = np.zeros(1, dtype=np.int64)
        fb = np.zeros(1)
        _check(load().fc2_stage_times(self.h, ms.ctypes.data, nl.ctypes.data, fb.ctypes.data),
               "fc2_stage_times")
        return ms, int(nl[0]), float(fb[0])

    @property
    def t0(self):
        return float(load().fc2_debug_t0(self.h))

    def debug_fault(self, wait_cycles=0, drop_tile=-1):
        """Test-only fault injection (fc2_debug_fault): limit of the bulk-copy
        transform's waits in SM cycles (0 = default) and a tile whose copy is
        armed but never issued (-1 = none)."""
        _check(load().fc2_debug_fault(self.h, int(wait_cycles), int(drop_tile)),
               "fc2_debug_fault")

    def significance(self, log_p=None):
        """Significance of the last execute (fc2_significance): returns
        (log_p [H, N] or None, j_min [H], log_p_min [H], adj_scale [H]).
        log_p: True for a new host array, or a preallocated float64 numpy array
        or CUDA tensor of H*N elements; None skips the full array."""
        if log_p is True:
            log_p = np.empty((self.H, self.N), dtype=np.float64)
        jmin = np.zeros(self.H, dtype=np.int64)
        lpmin = np.zeros(self.H)
        adj = np.zeros(self.H)
        _check(load().fc2_significance(self.h, _ptr(log_p), jmin.ctypes.data, lpmin.ctypes.data,
                                       adj.ctypes.data), "fc2_significance")
        return log_p, jmin, lpmin, adj


def last_tier(tier=4):
    """Last tier of the mixed path's exact fix-up for the process (4 default,
    3 = double sums)."""
    load().fc2_debug_last_tier(int(tier))


def batch_timing(enable=True):
    """Stage timing of the batched path on or off (fc2_debug_batch_timing)."""
    load().fc2_debug_batch_timing(int(bool(enable)))


BATCH_STAGES = ("spread", "fft", "assemble", "fixup", "peaks")

# fc2_options.autotune: single-curve plans tune with 1 (True) only; the batched
# path tunes by default ("table": the tuning table or cache file, tuning on a
# miss), "retune" tunes anew, "fixed" keeps the default configuration
AUTOTUNE = {"fixed": -1, "table": 0, "retune": 1}
FFT_FAMILY_NAMES = {0: "radix-16 stages in shared memory", 1: "two register stages",
                    2: "radix-16 stages fed by bulk copies",
                    3: "two register stages of radix 32 (512 threads)",
                    4: "two register stages of radix 32 (512 threads), also 2^9 passes"}


def batch_config():
    """Launch configuration of the last batched call's last chunk
    (fc2_debug_batch_config) as a dict."""
    v = np.zeros(13, dtype=np.int64)
    load().fc2_debug_batch_config(v.ctypes.data)
    npass = int(v[5])
    return dict(source=("fixed", "table", "tuned")[int(v[0])] if 0 <= v[0] <= 2 else int(v[0]),
                fft_family=FFT_FAMILY_NAMES.get(int(v[1]), int(v[1])),
                fft_log2_radices=[int(r) for r in v[6:6 + npass]],
                spread_tile=int(v[2]), assemble_block=int(v[3]), exact_item_samples=int(v[4]),
                transform_group=int(v[12]), configurations_timed=int(v[10]),
                tuning_ms=float(v[11:12].view(np.float64)[0]))


def batch_force(spread_tile=0, assemble_block=0, exact_item_samples=0, transform_group=0):
    """Fixed configuration of batched calls that do not tune (autotune
    "fixed" or a transform family requested); zeros keep the defaults."""
    load().fc2_debug_batch_force(int(spread_tile), int(assemble_block), int(exact_item_samples),
                                 int(transform_group))


def batch_force_plan(radices=(), family=1):
    """Fixed transform plan (log2 radices, first pass first) and float kernel
    family (0 radix-16 shared memory, 1 register stages, 2 bulk copies) of
    batched calls that do not tune; () clears it."""
    r = np.ascontiguousarray(radices, dtype=np.int32)
    load().fc2_debug_batch_force_plan(r.ctypes.data if r.size else None, int(r.size), int(family))


def batch_forget_tuning():
    """Empty the process's tuning table (the cache file is read again)."""
    load().fc2_debug_batch_forget_tuning()


def spread_force_general(on=True):
    """Send every spreading tile to the general kernel (True) or restore the
    default, where tiles of one sample set that fit one staging batch go to
    the single-batch kernel (False)."""
    load().fc2_debug_spread_force_general(int(bool(on)))


def trim_device_memory(device=0):
    """Return the library's cached device memory on `device` to the system."""
    _check(load().fc2_trim_device_memory(int(device)), "fc2_trim_device_memory")


def periodogram(t, x, sigma, H, f_min, df, N, oversample=2, prec="fp64", **kw):
    """One-shot: Delta chi^2 [H, N], best records, peak records, chi2_0."""
    with Plan(t, x, sigma, H, f_min, df, N, oversample, prec, **kw) as p:
        return p.execute()


def execute_batched(offsets, t, x, sigma, H, f_min, df, N, oversample=2, prec="mixed", top_k=8,
                    kernel_width=0, dchi2=None, stream=None, device=0, autotune=False,
                    fft_kernel="default", shared_sampling=False):
    """Many curves in one call (fc2_execute_batched).  offsets [C+1], t/x/sigma
    concatenated (numpy host arrays, or CUDA tensors -> read in place); H, f_min,
    df, N per curve.  dchi2: optional preallocated float32 output (numpy or
    CUDA tensor) of sum_c H_c N_c elements.  Returns (dchi2, peaks, stats dict);
    peaks[c][r] is record r of curve c as a dict (``BatchPeaks``)."""
    lib = load()
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    C = offsets.size - 1
    H = np.ascontiguousarray(np.broadcast_to(H, (C,)), dtype=np.int32)
    f_min = np.ascontiguousarray(np.broadcast_to(f_min, (C,)), dtype=np.float64)
    df = np.ascontiguousarray(np.broadcast_to(df, (C,)), dtype=np.float64)
    N = np.ascontiguousarray(np.broadcast_to(N, (C,)), dtype=np.int64)
    dev = _is_dev(t)
    if not dev:
        t = np.ascontiguousarray(t, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    total = int(np.sum(H.astype(np.int64) * N))
    if dchi2 is None:
        dchi2 = np.empty(total, dtype=np.float32)
    K = int(top_k or 8)
    peaks = np.zeros((C, K), dtype=BEST_DTYPE)
    opt = make_options(prec, kernel_width, K, 0.0, stream, device, inputs_on_device=dev,
                       autotune=autotune, fft_kernel=fft_kernel, shared_sampling=shared_sampling)
    rc = lib.fc2_execute_batched(C, offsets.ctypes.data, _ptr(t), _ptr(x), _ptr(sigma),
                                 H.ctypes.data, f_min.ctypes.data, df.ctypes.data, N.ctypes.data,
                                 int(oversample), ctypes.byref(opt), _ptr(dchi2),
                                 peaks.ctypes.data)
    _check(rc, "fc2_execute_batched")
    st = np.zeros(5, dtype=np.int64)
    lib.fc2_debug_batch_counts(st.ctypes.data)
    ph = np.zeros(7)
    lib.fc2_debug_batch_phase_ms(ph.ctypes.data)
    sm = np.zeros(6)
    lib.fc2_debug_batch_stage_ms(sm.ctypes.data)
    return dchi2, BatchPeaks(peaks), dict(launches=int(lib.fc2_debug_batch_launches()),
                             resolved=int(st[0]), exact=int(st[1]),
                             exact_double_float=int(st[2]), exact_double=int(st[3]),
                             graphs=int(st[4]),
                             host_phase_ms=dict(zip(("setup", "alloc", "moments", "layout",
                                                     "graph", "wait", "release"),
                                                    (float(v) for v in ph))),
                             stage_ms=dict(zip(BATCH_STAGES, (float(v) for v in sm[:5]))),
                             fft_alg_bytes=float(sm[5]), config=batch_config())


def _backward_argtypes(lib):
    if getattr(lib, "_bw_ready", False):
        return
    lib.fc2_backward.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P, _P]
    lib.fc2_backward.restype = ctypes.c_int
    lib.fc2_backward_batched.argtypes = [ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P,
                                         ctypes.c_int, _P, _P, ctypes.POINTER(Options), _P, _P,
                                         _P, _P, _P]
    lib.fc2_backward_batched.restype = ctypes.c_int
    lib._bw_ready = True


def plan_backward(plan, peak_j, grad_out=None, want_samples=True):
    """fc2_backward on a Plan: exact gradients at the bins peak_j and Newton
    refinement.  Returns dict(f_refined, dchi2_refined, d_df [K], d_dx [K, n],
    d_dsigma [K, n]) as numpy arrays."""
    lib = load()
    _backward_argtypes(lib)
    pj = np.ascontiguousarray(peak_j, dtype=np.int64)
    K = pj.size
    g = None if grad_out is None else np.ascontiguousarray(grad_out, dtype=np.float64)
    fr, dr, dd = np.zeros(K), np.zeros(K), np.zeros(K)
    dx = np.zeros((K, plan.n)) if want_samples else None
    ds = np.zeros((K, plan.n)) if want_samples else None
    rc = lib.fc2_backward(plan.h, K, pj.ctypes.data, None if g is None else g.ctypes.data,
                          fr.ctypes.data, dr.ctypes.data, dd.ctypes.data,
                          None if dx is None else dx.ctypes.data,
                          None if ds is None else ds.ctypes.data)
    _check(rc, "fc2_backward")
    return dict(f_refined=fr, dchi2_refined=dr, d_df=dd, d_dx=dx, d_dsigma=ds)


Plan.backward = plan_backward


def backward_batched(offsets, t, x, sigma, H, f_min, df, N, peak_j, grad_out=None, stream=None,
                     device=0, d_dx=None, d_dsigma=None):
    """fc2_backward_batched: peak_j [C, K].  Returns dict of f_refined, dchi2_refined,
    d_df ([C, K]) and d_dx, d_dsigma (flat, curve c peak r at K*off[c] + r*n_c)."""
    lib = load()
    _backward_argtypes(lib)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    C = offsets.size - 1
    pj = np.ascontiguousarray(peak_j, dtype=np.int64).reshape(C, -1)
    K = pj.shape[1]
    H = np.ascontiguousarray(np.broadcast_to(H, (C,)), dtype=np.int32)
    f_min = np.ascontiguousarray(np.broadcast_to(f_min, (C,)), dtype=np.float64)
    df = np.ascontiguousarray(np.broadcast_to(df, (C,)), dtype=np.float64)
    N = np.ascontiguousarray(np.broadcast_to(N, (C,)), dtype=np.int64)
    dev = _is_dev(t)
    if not dev:
        t = np.ascontiguousarray(t, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    g = None if grad_out is None else np.ascontiguousarray(grad_out, dtype=np.float64)
    ntot = int(offsets[-1] - offsets[0])
    fr, dr, dd = np.zeros((C, K)), np.zeros((C, K)), np.zeros((C, K))
    if d_dx is None:
        d_dx = np.zeros(K * ntot)
    if d_dsigma is None:
        d_dsigma = np.zeros(K * ntot)
    opt = make_options("fp64", 0, K, 0.0, stream, device, inputs_on_device=dev)
    rc = lib.fc2_backward_batched(C, offsets.ctypes.data, _ptr(t), _ptr(x), _ptr(sigma),
                                  H.ctypes.data, f_min.ctypes.data, df.ctypes.data, N.ctypes.data,
                                  K, pj.ctypes.data, None if g is None else g.ctypes.data,
                                  ctypes.byref(opt), fr.ctypes.data, dr.ctypes.data,
                                  dd.ctypes.data, _ptr(d_dx), _ptr(d_dsigma))
    _check(rc, "fc2_backward_batched")
    return dict(f_refined=fr, dchi2_refined=dr, d_df=dd, d_dx=d_dx, d_dsigma=d_dsigma)


def peaks_function():
    """torch.autograd.Function: (x, sigma) -> Delta chi^2_H at the top-K peak
    bins of a fixed time grid; backward through fc2_backward (exact adjoint)."""
    import torch

    class Fchi2Peaks(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, sigma, t, H, f_min, df, N, oversample=2, prec="mixed", top_k=8):
            xn = x.detach().cpu().numpy().astype(np.float64)
            sn = sigma.detach().cpu().numpy().astype(np.float64)
            tn = np.asarray(t, dtype=np.float64)
            plan = Plan(tn, xn, sn, H, f_min, df, N, oversample, prec, top_k=top_k)
            _, _, peaks, _ = plan.execute()
            js = np.array([p["j"] for p in peaks if p["j"] >= 0], dtype=np.int64)
            vals = torch.tensor([p["dchi2"] for p in peaks if p["j"] >= 0], dtype=torch.float64)
            ctx.plan = plan
            ctx.js = js
            ctx.dev = x.device
            jt = torch.from_numpy(js).to(x.device)
            ctx.mark_non_differentiable(jt)
            return vals.to(x.device), jt

        @staticmethod
        def backward(ctx, g_vals, g_js):
            g = g_vals.detach().cpu().numpy().astype(np.float64)
            r = ctx.plan.backward(ctx.js, grad_out=g)
            gx = torch.from_numpy(r["d_dx"].sum(axis=0)).to(ctx.dev)
            gs = torch.from_numpy(r["d_dsigma"].sum(axis=0)).to(ctx.dev)
            ctx.plan.close()
            return gx, gs, None, None, None, None, None, None, None, None

    return Fchi2Peaks
