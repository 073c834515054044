"""The paper's own Fchi2 algorithm on the host (numpy): a CPU baseline.

TEST INFRASTRUCTURE: used by ``bench.py`` (the paper's method timed on the
host, with its transform / regression split, Sec. 4) and by the CPU tests.
It restates Sec. 3b-3c step by step, in double precision:

1. moments: w = sigma^-2, xbar = sum w x / sum w (Sec. 3b), chi2_0 (Sec. 3c);
2. gridding: weights and weighted data w (x - xbar) summed into the lower cell
   floor((t - T0) / dt) of zero-padded arrays of M cells, dt = 1 / (M df)
   (Kronecker delta, Sec. 3b; cells from ``oracle.paper_grid_times``);
3. one FFT of length M, sign e^{+i} (Eq. eqPQ), of the packed pair qhat + i phat;
   Qhat, Phat separated by the conjugate symmetry of real inputs;
4. per trial bin fhat = f_min / df + j: alpha from C', S' (real and imaginary
   parts of Qhat) at (h - h') fhat and (h + h') fhat, beta from Phat at h fhat
   (Sec. 2 Eqs. eqalphafirst..eqalpha and the beta equations), in the basis
   order constant, sin(h.), cos(h.) of Eq. eqtrunc;
5. one Cholesky factorisation of the (2H + 1)-square alpha per bin, z = L^-1 beta,
   Delta chi^2_{H'} = sum_{l=1}^{2H'} z_l^2 for every H' (the leading blocks of
   the factor are the factors of the nested models, Eq. eqchix); a column whose
   pivot is below 1e-13 of its diagonal is dropped (z_l = 0).

The factorisation runs column by column, each step over all bins at once.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import oracle

TAU = 1e-13


def _alpha_beta(Q, P, H):
    """alpha [nb, m, m], beta [nb, m] from Q[k], P[k] (k = 0..2H, arrays over
    bins; Q[-k] = conj Q[k])."""
    nb = Q[0].shape[0]
    m = 2 * H + 1

    def Cp(k):
        return Q[abs(k)].real

    def Sp(k):
        return Q[k].imag if k >= 0 else -Q[-k].imag

    A = np.empty((nb, m, m))
    A[:, 0, 0] = Cp(0)
    for h in range(1, H + 1):
        A[:, 0, 2 * h - 1] = A[:, 2 * h - 1, 0] = Sp(h)
        A[:, 0, 2 * h] = A[:, 2 * h, 0] = Cp(h)
        for hp in range(1, H + 1):
            A[:, 2 * h - 1, 2 * hp - 1] = 0.5 * (Cp(h - hp) - Cp(h + hp))
            A[:, 2 * h - 1, 2 * hp] = 0.5 * (Sp(h + hp) + Sp(h - hp))
            A[:, 2 * h, 2 * hp - 1] = 0.5 * (Sp(h + hp) - Sp(h - hp))
            A[:, 2 * h, 2 * hp] = 0.5 * (Cp(h - hp) + Cp(h + hp))
    B = np.empty((nb, m))
    B[:, 0] = P[0].real
    for h in range(1, H + 1):
        B[:, 2 * h - 1] = P[h].imag
        B[:, 2 * h] = P[h].real
    return A, B


def _nested_dchi2(A, B, H):
    """Cholesky of every alpha at once with the rank rule; returns [nb, H]."""
    nb, m, _ = A.shape
    L = np.zeros_like(A)
    z = np.zeros((nb, m))
    for l in range(m):
        d = A[:, l, l] - np.einsum("bk,bk->b", L[:, l, :l], L[:, l, :l])
        keep = d > TAU * A[:, l, l]
        piv = np.sqrt(np.where(keep, d, 1.0))
        L[:, l, l] = np.where(keep, piv, 0.0)
        for r in range(l + 1, m):
            v = A[:, r, l] - np.einsum("bk,bk->b", L[:, r, :l], L[:, l, :l])
            L[:, r, l] = np.where(keep, v / piv, 0.0)
        rhs = B[:, l] - np.einsum("bk,bk->b", L[:, l, :l], z[:, :l])
        z[:, l] = np.where(keep, rhs / piv, 0.0)
    zz = z[:, 1:] ** 2
    return np.stack([zz[:, :2 * h].sum(axis=1) for h in range(1, H + 1)], axis=1)


def fchi2_paper(t, x, sigma, H, f_min, df, bins, M, T0=None):
    """Delta chi^2 [len(bins), H] by the paper's method, and the seconds spent in
    (gridding, transform, regression).  f_min must be a whole number of df steps;
    M > 4 H (f_min / df + max bin) keeps every harmonic below M / 2."""
    t = np.asarray(t, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    bins = np.asarray(bins, dtype=np.int64)
    s0 = int(round(f_min / df))
    if abs(f_min / df - s0) > 1e-9 * max(1.0, f_min / df):
        raise ValueError("f_min must be a whole number of df steps")
    if 4 * H * (s0 + int(bins.max())) >= M:
        raise ValueError("M too small for the harmonics")
    tm0 = time.perf_counter()
    w = 1.0 / (sigma * sigma)
    W = math.fsum(w)
    xbar = math.fsum(w * x) / W
    cp = w * (x - xbar)
    T0 = t.min() if T0 is None else T0
    _, cells = oracle.paper_grid_times(t, T0, df, M)
    z = np.zeros(M, dtype=np.complex128)
    np.add.at(z, cells, w + 1j * cp)
    tm1 = time.perf_counter()
    Z = M * np.fft.ifft(z)  # sum_c z[c] e^{+2 pi i m c / M}
    tm2 = time.perf_counter()
    fh = s0 + bins
    Q, P = [], []
    for k in range(2 * H + 1):
        idx = (k * fh) % M
        zp, zm = Z[idx], np.conj(Z[(-idx) % M])
        Q.append(0.5 * (zp + zm))
        if k <= H:
            P.append(-0.5j * (zp - zm))
    A, B = _alpha_beta(Q, P, H)
    d = _nested_dchi2(A, B, H)
    tm3 = time.perf_counter()
    return d, {"grid_s": tm1 - tm0, "fft_s": tm2 - tm1, "solve_s": tm3 - tm2}
