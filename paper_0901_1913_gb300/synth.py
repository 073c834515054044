"""Seeded synthetic light curves shaped like the workloads the Fchi2 method targets.

This module only draws random inputs; it holds none of the periodogram's
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The paper's own test set (Hipparcos epoch photometry, Sec. 4) is not available;
these generators stand in for it with the shapes it describes: irregular,
season- and night-windowed sampling, heteroscedastic errors, periodic signals
with harmonic content, and pure-noise nulls.  Every stream comes from
numpy's PCG64 through ``SeedSequence``, so a (config, seed) pair always yields
the same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DAY_YEAR = 365.25


@dataclass
class Curve:
    t: np.ndarray
    x: np.ndarray
    sigma: np.ndarray
    H: int
    f_min: float
    df: float
    N: int
    oversample: int = 2
    truth: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.t.shape[0])


@dataclass
class Batch:
    """Curves packed in CSR form: samples of curve c are offsets[c]:offsets[c+1]."""
    offsets: np.ndarray
    t: np.ndarray
    x: np.ndarray
    sigma: np.ndarray
    H: np.ndarray
    f_min: np.ndarray
    df: np.ndarray
    N: np.ndarray
    oversample: int = 2
    truth: list = field(default_factory=list)

    @property
    def C(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def curve(self, c: int) -> Curve:
        a, b = int(self.offsets[c]), int(self.offsets[c + 1])
        return Curve(self.t[a:b], self.x[a:b], self.sigma[a:b], int(self.H[c]),
                     float(self.f_min[c]), float(self.df[c]), int(self.N[c]),
                     self.oversample, self.truth[c] if self.truth else {})


def _rng(seed: int, *spawn_path: int) -> np.random.Generator:
    """Stream of the child at `spawn_path` of SeedSequence(seed): the child k of
    a sequence has spawn key (parent key..., k), so it is built directly (the
    same bytes as spawning k + 1 children and taking the last)."""
    ss = np.random.SeedSequence(seed, spawn_key=tuple(int(k) for k in spawn_path))
    return np.random.Generator(np.random.PCG64(ss))


def lognormal_sigma(rng, n, median=0.05, s=0.4):
    return np.exp(math.log(median) + s * rng.standard_normal(n))


def seasonal_night_times(rng, n, T, season_on=182.6, half_window=1.0 / 6.0):
    """Times on random nights inside the 'on' half of each year, each within an
    8-hour window centred on local midnight (t = d + 0.5 +- 1/6 d)."""
    d = np.arange(int(math.ceil(T)), dtype=np.float64)  # whole days 0, 1, .. below T
    d = d[d < T]
    nights = d[np.fmod(d, DAY_YEAR) < season_on]
    pick = nights[rng.integers(0, nights.size, n)]
    t = pick + 0.5 + rng.uniform(-half_window, half_window, n)
    return np.sort(t)


def sawtooth(t, f0, amp, nh=8):
    s = np.zeros_like(t)
    for h in range(1, nh + 1):
        s += ((-1.0) ** (h + 1)) * np.sin(2 * np.pi * h * f0 * t) / h
    return amp * (2.0 / np.pi) * s


def gaussian_pulse(t, f0, amp, duty=0.1, phase0=0.0):
    ph = np.mod(f0 * t + phase0, 1.0) - 0.5
    width = duty / 2.355  # duty cycle read as the pulse FWHM in phase
    return amp * np.exp(-0.5 * (ph / width) ** 2)


# ----------------------------------------------------------------------------
# The five workloads.  Readings where the workload text is silent are marked
# "reading" and listed with the input recipe in the design notes.
# ----------------------------------------------------------------------------

def short_curve(seed: int = 0, n: int = 1000, N: int = 16384) -> Curve:
    """Single short curve: 1000 samples over 100 d minus two 10 d gaps, three
    harmonics of 1.37 /d, H = 3, N trial frequencies on [0.01, 10] /d."""
    rng = _rng(seed)
    t = np.empty(0)
    while t.size < n:
        cand = rng.uniform(0.0, 100.0, 2 * n)
        keep = ~(((cand >= 30.0) & (cand < 40.0)) | ((cand >= 65.0) & (cand < 75.0)))
        t = np.concatenate([t, cand[keep]])
    t = np.sort(t[:n])
    sigma = lognormal_sigma(rng, n)
    f0 = 1.37
    amps = (1.0, 0.4, 0.15)
    phases = rng.uniform(0.0, 2 * np.pi, 3)
    x = np.zeros(n)
    for h, (a, ph) in enumerate(zip(amps, phases), start=1):
        x += a * np.sin(2 * np.pi * h * f0 * t + ph)
    x += sigma * rng.standard_normal(n)
    f_min, f_max = 0.01, 10.0
    df = (f_max - f_min) / (N - 1)
    return Curve(t, x, sigma, 3, f_min, df, N, 2,
                 dict(f0=f0, amps=amps, phases=tuple(phases)))


def long_curve(seed: int = 2, n: int = 100_000, N: int = 1 << 22, T: float = 3000.0,
            f_max: float = 20.0, H: int = 6, oversample: int = 4) -> Curve:
    """Single long curve: seasonal (6 months on/off) nightly sampling over
    3000 d, 8-harmonic sawtooth at f0 = 0.7312 /d (reading) with
    rms(signal)/median(sigma) = 5 (reading of "SNR ~ 5"), H = 6,
    f_min = df = f_max / N, 4x oversampled grids."""
    rng = _rng(seed)
    t = seasonal_night_times(rng, n, T)
    sigma = lognormal_sigma(rng, n)
    f0 = 0.7312
    s = sawtooth(t, f0, 1.0)
    amp = 5.0 * np.median(sigma) / np.sqrt(np.mean(s * s))
    x = amp * s + sigma * rng.standard_normal(n)
    df = f_max / N
    return Curve(t, x, sigma, H, df, df, N, oversample, dict(f0=f0, amp=amp))


def _survey_curve(rng, n, T, H, f0, shape, snr, null):
    t = seasonal_night_times(rng, n, T)
    sigma = lognormal_sigma(rng, n)
    if null:
        sig = np.zeros(n)
    elif shape == 0:
        sig = np.sin(2 * np.pi * f0 * t + rng.uniform(0, 2 * np.pi))
    elif shape == 1:
        sig = sawtooth(t + rng.uniform(0, 1.0 / f0), f0, 1.0)
    else:
        sig = gaussian_pulse(t, f0, 1.0, 0.1, rng.uniform(0, 1))
    if not null:
        rms = np.sqrt(np.mean((sig - sig.mean()) ** 2))
        sig = sig * (snr * np.median(sigma) / max(rms, 1e-300))
    x = sig + sigma * rng.standard_normal(n)
    return t, x, sigma


def survey_batch(seed: int = 3, C: int = 4096, N: int = 1 << 18, T: float = 1000.0,
            f_max: float = 12.0, n_median: float = 2000.0, n_lo: int = 50,
            n_hi: int = 20000) -> Batch:
    """Batched survey: C curves, n_c ~ lognormal(median 2000, s = 1.0 reading)
    clipped to [50, 20000], H_c ~ U{2..6}, f0 ~ U[0.05, 10] /d, shapes
    sinusoid / sawtooth / Gaussian pulse (1/3 each), per-point SNR ~ U[0.5, 5]
    (reading), 30% pure-noise nulls; N = 2^18 per curve, f_min = df = 12/N."""
    top = _rng(seed)
    n_c = np.clip(np.round(np.exp(math.log(n_median) + 1.0 * top.standard_normal(C))),
                  n_lo, n_hi).astype(np.int64)
    Hs = top.integers(2, 7, C)
    f0s = top.uniform(0.05, 10.0, C)
    shapes = top.integers(0, 3, C)
    snrs = top.uniform(0.5, 5.0, C)
    nulls = top.uniform(0, 1, C) < 0.3
    ts, xs, ss, truth = [], [], [], []
    for c in range(C):
        rng = _rng(seed, c)
        t, x, s = _survey_curve(rng, int(n_c[c]), T, int(Hs[c]), f0s[c], shapes[c],
                                snrs[c], bool(nulls[c]))
        ts.append(t); xs.append(x); ss.append(s)
        truth.append(dict(f0=float(f0s[c]), shape=int(shapes[c]), null=bool(nulls[c])))
    offsets = np.zeros(C + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(n_c)
    df = f_max / N
    return Batch(offsets, np.concatenate(ts), np.concatenate(xs), np.concatenate(ss),
                 Hs.astype(np.int32), np.full(C, df), np.full(C, df),
                 np.full(C, N, dtype=np.int64), 2, truth)


def shared_field(seed: int = 6, C: int = 1024, n: int = 2000, N: int = 1 << 18,
                 T: float = 1000.0, f_max: float = 12.0, H: int = 4) -> Batch:
    """Many sources in one field (Sec. 4's shared sampling, reading): one
    seasonal/nightly cadence of n epochs over T days shared by all C sources,
    errors sigma_c = r_c sigma with one lognormal sigma per epoch and
    r_c ~ U[0.5, 2]; signals as the survey's (f0 ~ U[0.05, 10] /d, sinusoid /
    sawtooth / Gaussian pulse, per-point SNR ~ U[0.5, 5], 30% nulls); H = 4,
    N = 2^18, f_min = df = f_max / N."""
    top = _rng(seed)
    t = seasonal_night_times(top, n, T)
    sigma0 = lognormal_sigma(top, n)
    r = top.uniform(0.5, 2.0, C)
    f0s = top.uniform(0.05, 10.0, C)
    shapes = top.integers(0, 3, C)
    snrs = top.uniform(0.5, 5.0, C)
    nulls = top.uniform(0, 1, C) < 0.3
    xs, ss, truth = [], [], []
    for c in range(C):
        rng = _rng(seed, c)
        sigma = r[c] * sigma0
        if nulls[c]:
            sig = np.zeros(n)
        elif shapes[c] == 0:
            sig = np.sin(2 * np.pi * f0s[c] * t + rng.uniform(0, 2 * np.pi))
        elif shapes[c] == 1:
            sig = sawtooth(t + rng.uniform(0, 1.0 / f0s[c]), f0s[c], 1.0)
        else:
            sig = gaussian_pulse(t, f0s[c], 1.0, 0.1, rng.uniform(0, 1))
        if not nulls[c]:
            rms = np.sqrt(np.mean((sig - sig.mean()) ** 2))
            sig = sig * (snrs[c] * np.median(sigma) / max(rms, 1e-300))
        xs.append(sig + sigma * rng.standard_normal(n))
        ss.append(sigma)
        truth.append(dict(f0=float(f0s[c]), shape=int(shapes[c]), null=bool(nulls[c]),
                          r=float(r[c])))
    offsets = np.arange(C + 1, dtype=np.int64) * n
    df = f_max / N
    return Batch(offsets, np.tile(t, C), np.concatenate(xs), np.concatenate(ss),
                 np.full(C, H, dtype=np.int32), np.full(C, df), np.full(C, df),
                 np.full(C, N, dtype=np.int64), 2, truth)


def adjoint_batch(seed: int = 4, C: int = 1024, n: int = 2000, N: int = 1 << 16,
            T: float = 500.0, f_max: float = 12.0, H: int = 4) -> Batch:
    """Differentiation batch: C curves of n = 2000 samples over a seasonal
    500 d (reading), H = 4, N = 2^16, signals as the non-null survey curves."""
    top = _rng(seed)
    f0s = top.uniform(0.05, 10.0, C)
    shapes = top.integers(0, 3, C)
    snrs = top.uniform(0.5, 5.0, C)
    ts, xs, ss, truth = [], [], [], []
    for c in range(C):
        rng = _rng(seed, c)
        t, x, s = _survey_curve(rng, n, T, H, f0s[c], shapes[c], snrs[c], False)
        ts.append(t); xs.append(x); ss.append(s)
        truth.append(dict(f0=float(f0s[c]), shape=int(shapes[c]), null=False))
    offsets = np.arange(C + 1, dtype=np.int64) * n
    df = f_max / N
    return Batch(offsets, np.concatenate(ts), np.concatenate(xs), np.concatenate(ss),
                 np.full(C, H, dtype=np.int32), np.full(C, df), np.full(C, df),
                 np.full(C, N, dtype=np.int64), 2, truth)


def large_curve(seed: int = 5, cadence_min: float = 2.0, years: float = 4.0,
            N: int = 1 << 26, f_max: float = 24.0, H: int = 8,
            dropout: float = 0.05, oversample: int = 2) -> Curve:
    """Large single curve: regular cadence (2 min by default, reading; 30 min
    for the exact-alias variant) over 4 years with 5% random dropouts; sigma is
    a two-level mixture 0.001 (p = 0.8) / 0.01; three incommensurate periods
    with 4 harmonics each (a_h = A_s / h); AR(1) red noise rho = 0.9 with
    stationary std 0.003; H = 8, f_min = df = 24 / N."""
    rng = _rng(seed)
    step = cadence_min / (24.0 * 60.0)
    slots = int(math.floor(years * DAY_YEAR / step))
    keep = rng.uniform(0, 1, slots) >= dropout
    t = np.arange(slots, dtype=np.float64)[keep] * step
    n = t.size
    sigma = np.where(rng.uniform(0, 1, n) < 0.8, 0.001, 0.01)
    fs = (0.4171, 1.3313, 3.0870)
    As = (0.01, 0.005, 0.003)
    x = np.zeros(n)
    for f, A in zip(fs, As):
        for h in range(1, 5):
            x += (A / h) * np.sin(2 * np.pi * h * f * t + rng.uniform(0, 2 * np.pi))
    rho, sd = 0.9, 0.003
    e = rng.standard_normal(n) * sd * math.sqrt(1 - rho * rho)
    e[0] = rng.standard_normal() * sd  # stationary start
    red = _ar1(e, rho)
    x += red + sigma * rng.standard_normal(n)
    df = f_max / N
    return Curve(t, x, sigma, H, df, df, N, oversample, dict(fs=fs, As=As))


def _ar1(e, rho):
    from scipy.signal import lfilter
    return lfilter([1.0], [1.0, -rho], e)


def tiny_curve(seed: int, n: int, T: float = 10.0, H: int = 2, N: int = 64,
               f_min: float = 0.05, df: float = 0.037, signal: float = 1.0) -> Curve:
    """Small irregular curve for exhaustive checks."""
    rng = _rng(seed)
    t = np.sort(rng.uniform(0.0, T, n))
    sigma = lognormal_sigma(rng, n, 0.3, 0.5)
    x = signal * np.sin(2 * np.pi * 0.71 * t + 0.3) + sigma * rng.standard_normal(n) + 2.0
    return Curve(t, x, sigma, H, f_min, df, N, 2)
