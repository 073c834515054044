"""ctypes front end of the C oracle (``fc2_oracle.c``).

TEST INFRASTRUCTURE: the oracle computes Delta chi^2 of the truncated Fourier
model (Palmer 2009, Sec. 1 Eq. "eqtrunc", Sec. 2 Eqs. "eqchigen", "eqchix")
directly from the samples -- Householder least squares per trial frequency and
per H', no FFT, no gridding.  The C file's header states each definition used.

``build()`` compiles the C file with gcc into ``oracle/_build``.  The calls here
only marshal arrays; threads split the trial bins across host cores (ctypes
releases the GIL during the foreign call, and the C code is re-entrant).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fc2_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libfc2_oracle.so")
_lib = None
_lock = threading.Lock()

TAU_R = 1e-10  # rank rule: drop a column whose residual norm < TAU_R * its norm

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.fc2o_moments.argtypes = [_D, _D, _D, i64, _D]
            lib.fc2o_dchi2_freqs.argtypes = [_D, _D, _D, i64, i32, _D, i64, dbl, _D, _D]
            lib.fc2o_dchi2_bins.argtypes = [_D, _D, _D, i64, i32, dbl, dbl, _I64, i64, dbl, _D, _D]
            lib.fc2o_coeffs.argtypes = [_D, _D, _D, i64, i32, dbl, dbl, _D, _D]
            lib.fc2o_trig_sums.argtypes = [_D, _D, i64, _D, i64, _D, _D]
            lib.fc2o_normal_eq.argtypes = [_D, _D, _D, i64, i32, dbl, _D, _D]
            lib.fc2o_grad.argtypes = [_D, _D, _D, i64, i32, dbl, dbl, _D, _D, _D, _D]
            lib.fc2o_refine.argtypes = [_D, _D, _D, i64, i32, dbl, dbl, dbl, dbl, _D, _D]
            lib.fc2o_dchi2_trend_freqs.argtypes = [_D, _D, _D, i64, i32, i32, _D, i64, dbl, _D,
                                                   _D, _D]
            for fn in ("fc2o_moments", "fc2o_dchi2_freqs", "fc2o_dchi2_bins", "fc2o_coeffs",
                       "fc2o_trig_sums", "fc2o_normal_eq", "fc2o_grad", "fc2o_refine",
                       "fc2o_dchi2_trend_freqs"):
                getattr(lib, fn).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def moments(x, sigma):
    """(W, xbar, chi2_0, sum w (x - xbar)) -- Sec. 3b and 3c definitions."""
    lib = _load()
    x, sigma = _f64(x), _f64(sigma)
    out = np.zeros(4)
    _check(lib.fc2o_moments(None, _p(x), _p(sigma), x.size, _p(out)), "moments")
    return tuple(float(v) for v in out)


def _threads(threads):
    if threads is None or threads <= 0:
        return os.cpu_count() or 1
    return threads


def dchi2_freqs(t, x, sigma, H, freqs, threads=None, tau_r=TAU_R, with_pivots=False):
    """Delta chi^2_{H'} for H' = 1..H at each frequency: array [len(freqs), H]."""
    lib = _load()
    t, x, sigma, freqs = _f64(t), _f64(x), _f64(sigma), _f64(np.atleast_1d(freqs))
    nf = freqs.size
    out = np.zeros((nf, H))
    piv = np.zeros((nf, H))
    nt = max(1, min(_threads(threads), nf))
    chunks = np.array_split(np.arange(nf), nt)

    def run(idx):
        if idx.size == 0:
            return 0
        fr = np.ascontiguousarray(freqs[idx])
        o = np.zeros((idx.size, H))
        pv = np.zeros((idx.size, H))
        rc = lib.fc2o_dchi2_freqs(_p(t), _p(x), _p(sigma), t.size, H, _p(fr), idx.size,
                                  tau_r, _p(o), _p(pv))
        out[idx] = o
        piv[idx] = pv
        return rc

    if nt == 1:
        rcs = [run(chunks[0])]
    else:
        with ThreadPoolExecutor(nt) as ex:
            rcs = list(ex.map(run, chunks))
    for rc in rcs:
        _check(rc, "dchi2")
    return (out, piv) if with_pivots else out


def freq_of(f_min, df, j):
    """Trial frequency f_j = f_min + j * df, evaluated in double exactly so."""
    return f_min + np.asarray(j, dtype=np.float64) * df


def dchi2_bins(t, x, sigma, H, f_min, df, bins, threads=None, tau_r=TAU_R, with_pivots=False):
    return dchi2_freqs(t, x, sigma, H, freq_of(f_min, df, np.asarray(bins, dtype=np.int64)),
                       threads=threads, tau_r=tau_r, with_pivots=with_pivots)


def dchi2_trend_freqs(t, x, sigma, H, D, freqs, threads=None, tau_r=TAU_R, with_pivots=False):
    """Trend fitted jointly with the harmonics (Sec. 4's polynomial detrending
    read as a joint fit): Delta chi^2_{H'} = chi^2(degree-D polynomial) -
    chi^2(polynomial + H' harmonics) at each frequency: ([len(freqs), H],
    chi2 of the polynomial alone[, minimum relative pivots])."""
    lib = _load()
    t, x, sigma, freqs = _f64(t), _f64(x), _f64(sigma), _f64(np.atleast_1d(freqs))
    nf = freqs.size
    out = np.zeros((nf, H))
    piv = np.zeros((nf, H))
    chi0 = np.zeros(1)
    nt = max(1, min(_threads(threads), nf))
    chunks = np.array_split(np.arange(nf), nt)

    def run(idx):
        fr = np.ascontiguousarray(freqs[idx])
        o = np.zeros((idx.size, H))
        pv = np.zeros((idx.size, H))
        c0 = np.zeros(1)
        rc = lib.fc2o_dchi2_trend_freqs(_p(t), _p(x), _p(sigma), t.size, H, int(D), _p(fr),
                                        idx.size, tau_r, _p(o), _p(pv), _p(c0))
        out[idx] = o
        piv[idx] = pv
        return rc, c0[0]

    if nt == 1:
        res = [run(chunks[0])]
    else:
        with ThreadPoolExecutor(nt) as ex:
            res = list(ex.map(run, chunks))
    for rc, _ in res:
        _check(rc, "dchi2_trend")
    chi0[0] = res[0][1]
    return (out, float(chi0[0]), piv) if with_pivots else (out, float(chi0[0]))


def dchi2_trend_bins(t, x, sigma, H, D, f_min, df, bins, threads=None, tau_r=TAU_R,
                     with_pivots=False):
    return dchi2_trend_freqs(t, x, sigma, H, D, freq_of(f_min, df, np.asarray(bins, dtype=np.int64)),
                             threads=threads, tau_r=tau_r, with_pivots=with_pivots)


def coeffs(t, x, sigma, Hp, f, tau_r=TAU_R):
    """(A[2Hp+1] absolute frame with xbar added to A0, Delta chi^2)."""
    lib = _load()
    t, x, sigma = _f64(t), _f64(x), _f64(sigma)
    A = np.zeros(2 * Hp + 1)
    d = np.zeros(1)
    _check(lib.fc2o_coeffs(_p(t), _p(x), _p(sigma), t.size, Hp, float(f), tau_r, _p(A), _p(d)),
           "coeffs")
    return A, float(d[0])


def trig_sums(t, c, freqs):
    """sum_i c_i exp(+i 2 pi f t_i) for each f (Sec. 2, Eq. eqPQ)."""
    lib = _load()
    t, c, freqs = _f64(t), _f64(c), _f64(np.atleast_1d(freqs))
    re = np.zeros(freqs.size)
    im = np.zeros(freqs.size)
    _check(lib.fc2o_trig_sums(_p(t), _p(c), t.size, _p(freqs), freqs.size, _p(re), _p(im)),
           "trig_sums")
    return re + 1j * im


def normal_eq(t, x, sigma, H, f):
    """(alpha [(2H+1)^2], beta [2H+1]) by direct sums over samples (Sec. 2)."""
    lib = _load()
    t, x, sigma = _f64(t), _f64(x), _f64(sigma)
    m = 2 * H + 1
    a = np.zeros((m, m))
    b = np.zeros(m)
    _check(lib.fc2o_normal_eq(_p(t), _p(x), _p(sigma), t.size, H, float(f), _p(a), _p(b)),
           "normal_eq")
    return a, b


def grad(t, x, sigma, H, f, tau_r=TAU_R):
    """(Delta chi^2_H, d/df, d/dx[n], d/dsigma[n]) at fixed f."""
    lib = _load()
    t, x, sigma = _f64(t), _f64(x), _f64(sigma)
    d = np.zeros(1)
    g = np.zeros(1)
    gx = np.zeros(t.size)
    gs = np.zeros(t.size)
    _check(lib.fc2o_grad(_p(t), _p(x), _p(sigma), t.size, H, float(f), tau_r, _p(d), _p(g),
                         _p(gx), _p(gs)), "grad")
    return float(d[0]), float(g[0]), gx, gs


def refine(t, x, sigma, H, a, b, tol=1e-12, tau_r=TAU_R):
    """Brent maximum of the exact Delta chi^2_H(f) on [a, b]: (f*, value)."""
    lib = _load()
    t, x, sigma = _f64(t), _f64(x), _f64(sigma)
    fs = np.zeros(1)
    v = np.zeros(1)
    _check(lib.fc2o_refine(_p(t), _p(x), _p(sigma), t.size, H, float(a), float(b), float(tol),
                           tau_r, _p(fs), _p(v)), "refine")
    return float(fs[0]), float(v[0])


def periodogram(t, x, sigma, H, f_min, df, N, threads=None, tau_r=TAU_R, with_pivots=False):
    """Full oracle periodogram over all N bins: [N, H] (small cases only)."""
    return dchi2_bins(t, x, sigma, H, f_min, df, np.arange(N), threads=threads, tau_r=tau_r,
                      with_pivots=with_pivots)


def chi2_logsf_even(x, Hp):
    """ln P(chi^2 with 2 Hp degrees of freedom >= x) -- the cumulative chi^2
    distribution of Sec. 3d's p(f) for a model with 2 Hp extra parameters.

    For an even number of degrees of freedom the survival function is the
    finite Poisson sum  e^{-y} sum_{i=0}^{Hp-1} y^i / i!,  y = x / 2, written
    out here term by term in log space (log-sum-exp over the terms).  x <= 0
    gives 0 (probability 1)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.maximum(x, 0.0) / 2.0
    out = np.zeros_like(y)
    pos = y > 0
    yp = y[pos]
    logs = np.stack([i * np.log(yp) - math.lgamma(i + 1) for i in range(int(Hp))])
    m = logs.max(axis=0)
    out[pos] = -yp + m + np.log(np.exp(logs - m).sum(axis=0))
    return out


def fhat(f_min, df, bins):
    """Trial count 'so far' at f_j (Sec. 3d): f_j / df, the index of f_j on a
    grid of spacing df that starts at 0, taken as at least 1."""
    f = freq_of(f_min, df, np.asarray(bins, dtype=np.int64))
    return np.maximum(f / df, 1.0)


def log_false_alarm(dchi2, f_min, df, bins):
    """ln p(f_j) = ln fhat_j + ln P_{2H', >= Delta chi^2}(Delta chi^2_{H'}(f_j))
    (Sec. 3d), for dchi2 [len(bins), H] (columns H' = 1..H)."""
    d = np.asarray(dchi2, dtype=np.float64)
    lf = np.log(fhat(f_min, df, bins))
    out = np.empty_like(d)
    for h in range(d.shape[1]):
        out[:, h] = lf + chi2_logsf_even(d[:, h], h + 1)
    return out


def adjusted_scale(dchi2_best, chi2_0, n):
    """Factor s_{H'} with Delta chi^2_adj = s_{H'} Delta chi^2 (Sec. 3d's adjusted
    Delta chi^2): the denominator is the best fit's residual chi^2 per degree of
    freedom, (chi2_0 - Delta chi^2_best) / (n - 2H' - 1)."""
    b = np.asarray(dchi2_best, dtype=np.float64)
    Hs = np.arange(1, b.size + 1)
    return (n - 2 * Hs - 1) / (chi2_0 - b)


def paper_grid_times(t, T0, df, M):
    """Sec. 3b's gridding, t_hat = floor((t - T0) / dt) with dt = 1 / (M df):
    the sample times moved to the lower edge of their cell of an array of M
    cells, returned relative to T0 as t_hat * dt (the array wraps with period
    M dt = 1 / df, which no trial frequency f_min + j df, f_min a multiple of
    df, can tell apart).  t - T0 is rounded to double as the library does;
    the cell index is then exact (rational arithmetic)."""
    from fractions import Fraction
    tau = np.asarray(t, dtype=np.float64) - np.float64(T0)
    fdf = Fraction(float(df))
    cells = np.empty(tau.size, dtype=np.int64)
    for i, v in enumerate(tau.tolist()):
        u = fdf * Fraction(v)
        frac = u - (u.numerator // u.denominator)
        cells[i] = (frac * int(M)).__floor__()
    return cells / (float(M) * float(df)), cells


def detrend(t, x, sigma, degree):
    """x minus its weighted least-squares polynomial of the given degree in t
    (weights sigma^-2): the polynomial detrending of the reference
    implementation described in Sec. 4 ("detrend the data with a polynomial
    fit ... removing variation out to t^3").  The fit is a library least-squares
    solve on the design 1, u, .., u^degree with u = (t - t_c) / s, t_c and s the
    centre and half-width of the time span (a change of basis only)."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sw = 1.0 / np.asarray(sigma, dtype=np.float64)
    lo, hi = t.min(), t.max()
    s = 0.5 * (hi - lo) if hi > lo else 1.0
    u = (t - 0.5 * (hi + lo)) / s
    D = np.vander(u, int(degree) + 1, increasing=True)
    c, *_ = np.linalg.lstsq(D * sw[:, None], x * sw, rcond=None)
    return x - D @ c
