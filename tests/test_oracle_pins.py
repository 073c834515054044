"""Pins of the CPU oracle to things other than itself (runs without a GPU).

Each test fixes the oracle against an independent fact: a library least-squares
solve, a published closed form, the paper's printed H = 2 layout, an exact
distribution, finite differences, or an exact invariance.  A plausible slip in
the oracle (a dropped harmonic, a sign of sin, an index of M_l, a transposed
alpha, a wrong weight power) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_0901_1913_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def design(t, f, Hp):
    D = np.ones((t.size, 2 * Hp + 1))
    for h in range(1, Hp + 1):
        D[:, 2 * h - 1] = np.sin(2 * np.pi * h * f * t)
        D[:, 2 * h] = np.cos(2 * np.pi * h * f * t)
    return D


def lstsq_dchi2(t, x, sigma, f, Hp):
    """chi2_0 - min_A sum w (x - D A)^2 with numpy's SVD least squares."""
    sw = 1.0 / sigma
    w = sw * sw
    xbar = np.sum(w * x) / np.sum(w)
    chi0 = np.sum(w * (x - xbar) ** 2)
    D = design(t, f, Hp) * sw[:, None]
    A, *_ = np.linalg.lstsq(D, x * sw, rcond=1e-12)
    return chi0 - np.sum((x * sw - D @ A) ** 2), chi0


# ------------------------------------------------------------------ moments

def test_moments_hand_example(oracle_mod):
    W, xbar, chi0, s1 = oracle_mod.moments([1.0, 3.0, 5.0], [1.0, 1.0, 0.5])
    # w = (1, 1, 4): W = 6, xbar = (1 + 3 + 20) / 6 = 4, chi0 = 9 + 1 + 4 = 14
    assert W == pytest.approx(6.0, rel=1e-15)
    assert xbar == pytest.approx(4.0, rel=1e-15)
    assert chi0 == pytest.approx(14.0, rel=1e-15)
    assert abs(s1) < 1e-14


# ------------------------------------------------------- brute force (lstsq)

@pytest.mark.parametrize("n", [5, 8, 13, 30, 64])
@pytest.mark.parametrize("H", [1, 2, 3])
def test_dchi2_matches_lstsq(oracle_mod, n, H):
    c = synth.tiny_curve(100 + n, n, H=H)
    rng = np.random.default_rng(n * 7 + H)
    freqs = np.concatenate([[0.71, 1.42], rng.uniform(0.05, 3.0, 6)])
    got = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, H, freqs, threads=1)
    for k, f in enumerate(freqs):
        for Hp in range(1, H + 1):
            ref, chi0 = lstsq_dchi2(c.t, c.x, c.sigma, f, Hp)
            assert abs(got[k, Hp - 1] - ref) <= 1e-10 * chi0, (n, H, f, Hp)


def test_underdetermined_fit_is_perfect(oracle_mod):
    # n = 4 samples, H' = 2 has 5 parameters: the fit is exact, Delta = chi2_0
    c = synth.tiny_curve(7, 4, H=2)
    got = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 2, [0.9])
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    assert got[0, 1] == pytest.approx(chi0, rel=1e-10)


# ------------------------------------------------- normal equations / sums

def test_trig_sums_match_library_fft(oracle_mod):
    # uniform times t_i = i / L: sum_i c_i e^{+2 pi i k t_i} = L * ifft(c)[k]
    L = 64
    rng = np.random.default_rng(3)
    c = rng.standard_normal(L)
    t = np.arange(L) / L
    ks = np.arange(L)
    got = oracle_mod.trig_sums(t, c, ks.astype(float))
    ref = L * np.fft.ifft(c)
    np.testing.assert_allclose(got, ref, atol=1e-12 * np.sum(np.abs(c)))
    # negative frequency is the complex conjugate (real weights)
    neg = oracle_mod.trig_sums(t, c, -ks[1:].astype(float))
    np.testing.assert_allclose(neg, np.conj(ref[1:]), atol=1e-12 * np.sum(np.abs(c)))


@pytest.mark.parametrize("H", [1, 3, 5])
def test_alpha_beta_from_trig_identities(oracle_mod, H):
    """Direct alpha/beta == assembly from C', S' at (h +- h') f and C, S at h f
    (Sec. 2, Eqs. eqalphafirst..eqalpha and the beta equations)."""
    c = synth.tiny_curve(11, 50, H=H)
    f = 0.613
    alpha, beta = oracle_mod.normal_eq(c.t, c.x, c.sigma, H, f)
    w = 1.0 / c.sigma ** 2
    _, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    ks = np.arange(-2 * H, 2 * H + 1)
    Q = dict(zip(ks, oracle_mod.trig_sums(c.t, w, ks * f)))
    P = dict(zip(ks, oracle_mod.trig_sums(c.t, w * (c.x - xbar), ks * f)))
    Cp = lambda k: Q[k].real  # noqa: E731
    Sp = lambda k: Q[k].imag  # noqa: E731
    m = 2 * H + 1
    A = np.zeros((m, m))
    A[0, 0] = Cp(0)
    for h in range(1, H + 1):
        A[0, 2 * h - 1] = A[2 * h - 1, 0] = Sp(h)
        A[0, 2 * h] = A[2 * h, 0] = Cp(h)
        for hp in range(1, H + 1):
            A[2 * h - 1, 2 * hp - 1] = 0.5 * (Cp(h - hp) - Cp(h + hp))
            A[2 * h - 1, 2 * hp] = 0.5 * (Sp(h + hp) + Sp(h - hp))
            A[2 * h, 2 * hp - 1] = 0.5 * (Sp(h + hp) - Sp(h - hp))
            A[2 * h, 2 * hp] = 0.5 * (Cp(h - hp) + Cp(h + hp))
    B = np.zeros(m)
    B[0] = P[0].real
    for h in range(1, H + 1):
        B[2 * h - 1] = P[h].imag
        B[2 * h] = P[h].real
    scale = np.sum(w)
    np.testing.assert_allclose(alpha, A, atol=1e-12 * scale)
    np.testing.assert_allclose(beta, B, atol=1e-12 * np.sum(w * np.abs(c.x - xbar)))
    # and beta^T alpha^-1 beta (Eq. eqchix) equals the QR Delta chi^2 of H' = H
    d = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, H, [f])[0, H - 1]
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    assert beta @ np.linalg.solve(alpha, beta) == pytest.approx(d, abs=1e-9 * chi0)


def _parse_terms(s):
    import re
    return [(float(cf), kind, int(k)) for cf, kind, k in re.findall(r"([+-]\d+)([RI])(\d+)", s)]


def _eval_terms(terms, spec):
    return sum(cf * (spec[k].real if kind == "R" else spec[k].imag) for cf, kind, k in terms)


def test_paper_h2_layout_golden(oracle_mod):
    """The paper's printed H = 2 alpha/beta (Sec. 3c), as corrected, equals the
    oracle's direct sums; the typeset version is wrong exactly where noted."""
    c = synth.tiny_curve(5, 60, H=2)
    f = 0.4377
    alpha, beta = oracle_mod.normal_eq(c.t, c.x, c.sigma, 2, f)
    w = 1.0 / c.sigma ** 2
    _, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    Q = oracle_mod.trig_sums(c.t, w, np.arange(5) * f)
    P = oracle_mod.trig_sums(c.t, w * (c.x - xbar), np.arange(5) * f)
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "alpha_h2_layout.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 25
    wrong = set()
    for r, col, printed, corrected in rows:
        r, col = int(r), int(col)
        val_c = 0.5 * _eval_terms(_parse_terms(corrected), Q)
        val_p = 0.5 * _eval_terms(_parse_terms(printed), Q)
        assert val_c == pytest.approx(alpha[r, col], abs=1e-12 * np.sum(w)), (r, col)
        if abs(val_p - alpha[r, col]) > 1e-6 * np.sum(w):
            wrong.add((r, col))
    assert wrong == {(1, 4), (4, 1), (2, 3), (3, 2)}
    brows = [ln.split() for ln in open(os.path.join(GOLDEN, "beta_h2_layout.txt"))
             if ln.strip() and not ln.startswith("#")]
    for idx, term in brows:
        assert _eval_terms(_parse_terms(term), P) == pytest.approx(
            beta[int(idx)], abs=1e-12 * np.sum(w * np.abs(c.x - xbar)))


# --------------------------------------------------------- closed forms

def gls_power(t, y, sigma, f):
    """Generalised (floating-mean) Lomb-Scargle power of Zechmeister & Kuerster
    (2009, A&A 496, 577), written from their published definitions."""
    wt = 1.0 / sigma ** 2
    wt = wt / wt.sum()
    om = 2 * np.pi * f
    cs, sn = np.cos(om * t), np.sin(om * t)
    Y, C, S = np.sum(wt * y), np.sum(wt * cs), np.sum(wt * sn)
    YY = np.sum(wt * y * y) - Y * Y
    YC = np.sum(wt * y * cs) - Y * C
    YS = np.sum(wt * y * sn) - Y * S
    CC = np.sum(wt * cs * cs) - C * C
    SS = np.sum(wt * sn * sn) - S * S
    CS = np.sum(wt * cs * sn) - C * S
    D = CC * SS - CS * CS
    return (SS * YC * YC + CC * YS * YS - 2 * CS * YC * YS) / (YY * D)


def test_h1_equals_generalised_lomb_scargle(oracle_mod):
    c = synth.short_curve(n=300, N=512)
    freqs = np.linspace(0.05, 5.0, 41)
    got = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 1, freqs)[:, 0]
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    ref = np.array([gls_power(c.t, c.x, c.sigma, f) for f in freqs]) * chi0
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-10 * chi0)


def test_noiseless_multiharmonic_recovers_signal(oracle_mod):
    rng = np.random.default_rng(1)
    n = 200
    t = np.sort(rng.uniform(0, 50, n))
    sigma = rng.uniform(0.5, 2.0, n)
    f_min, df = 0.1, 0.013
    j0 = 77
    f0 = f_min + j0 * df
    amps = [0.9, 0.5, 0.2]
    phis = [0.3, 1.9, -2.2]
    mean = 3.5
    x = mean + sum(a * np.sin(2 * np.pi * h * f0 * t + p)
                   for h, (a, p) in enumerate(zip(amps, phis), start=1))
    d = oracle_mod.dchi2_bins(t, x, sigma, 4, f_min, df, [j0])[0]
    _, _, chi0, _ = oracle_mod.moments(x, sigma)
    assert d[2] == pytest.approx(chi0, rel=1e-10)
    assert d[3] == pytest.approx(chi0, rel=1e-10)
    assert d[1] < chi0 * (1 - 1e-3)  # H' = 2 cannot fit the 3rd harmonic
    A, dd = oracle_mod.coeffs(t, x, sigma, 3, f0)
    assert A[0] == pytest.approx(mean, abs=1e-10)
    for h, (a, p) in enumerate(zip(amps, phis), start=1):
        # a sin(th + p) = a cos p sin th + a sin p cos th
        assert A[2 * h - 1] == pytest.approx(a * math.cos(p), abs=1e-10)
        assert A[2 * h] == pytest.approx(a * math.sin(p), abs=1e-10)


# ------------------------------------------------------------- invariants

@pytest.fixture(scope="module")
def inv_case():
    c = synth.tiny_curve(21, 120, T=30.0, H=4)
    freqs = np.concatenate([[0.71], np.random.default_rng(4).uniform(0.02, 4.0, 15)])
    return c, freqs


def test_bounds_and_monotone_in_H(oracle_mod, inv_case):
    c, freqs = inv_case
    d = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 4, freqs)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    assert np.all(d >= -1e-10 * chi0)
    assert np.all(d <= chi0 * (1 + 1e-12))
    assert np.all(np.diff(d, axis=1) >= -1e-9 * chi0)


def test_time_shift_invariance(oracle_mod, inv_case):
    c, freqs = inv_case
    a = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 4, freqs)
    b = oracle_mod.dchi2_freqs(c.t + 1234.5678, c.x, c.sigma, 4, freqs)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    np.testing.assert_allclose(a, b, atol=1e-8 * chi0)


def test_affine_and_sigma_scaling(oracle_mod, inv_case):
    c, freqs = inv_case
    a = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 4, freqs)
    b = oracle_mod.dchi2_freqs(c.t, -2.5 * c.x + 7.0, c.sigma, 4, freqs)
    s = oracle_mod.dchi2_freqs(c.t, c.x, 3.0 * c.sigma, 4, freqs)
    np.testing.assert_allclose(b, 6.25 * a, rtol=1e-10, atol=1e-10 * a.max())
    np.testing.assert_allclose(s, a / 9.0, rtol=1e-10, atol=1e-10 * a.max())


def test_permutation_invariance(oracle_mod, inv_case):
    c, freqs = inv_case
    p = np.random.default_rng(9).permutation(c.n)
    a = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, 4, freqs)
    b = oracle_mod.dchi2_freqs(c.t[p], c.x[p], c.sigma[p], 4, freqs)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-10 * a.max())


def test_exact_alias_rank_deficiency(oracle_mod):
    """30-min cadence: at h f = 24 /d the h-th sine vanishes on every sample;
    Delta chi^2 is the projection onto the span that remains (lstsq, SVD)."""
    rng = np.random.default_rng(2)
    t = np.arange(0, 400) / 48.0
    sigma = rng.uniform(0.5, 1.5, t.size)
    x = np.sin(2 * np.pi * 3.0 * t) + rng.standard_normal(t.size) * sigma
    f = 12.0  # h = 2 -> 24 /d: sin(2 pi 24 t) = sin(pi i) = 0
    d, piv = oracle_mod.dchi2_freqs(t, x, sigma, 3, [f], with_pivots=True)
    for Hp in (1, 2, 3):
        ref, chi0 = lstsq_dchi2(t, x, sigma, f, Hp)
        assert abs(d[0, Hp - 1] - ref) <= 1e-8 * chi0
    assert piv[0, 0] > 1e-3  # H' = 1 is well conditioned


# ------------------------------------------------------------- statistics

def test_gaussian_null_is_chi2_with_2H_dof(oracle_mod):
    """Under a constant source with Gaussian errors, Delta chi^2 at a fixed
    frequency follows chi^2 with 2H' degrees of freedom (Sec. 2)."""
    from scipy import stats
    rng = np.random.default_rng(123)
    n, R = 40, 3000
    t = np.sort(rng.uniform(0, 20, n))
    sigma = rng.uniform(0.3, 2.0, n)
    f = 0.537
    vals = np.empty((R, 3))
    for r in range(R):
        x = 5.0 + sigma * rng.standard_normal(n)
        vals[r] = oracle_mod.dchi2_freqs(t, x, sigma, 3, [f], threads=1)[0]
    for Hp in (1, 2, 3):
        k = 2 * Hp
        assert abs(vals[:, Hp - 1].mean() - k) < 4 * math.sqrt(2 * k / R)
        assert stats.kstest(vals[:, Hp - 1], stats.chi2(k).cdf).pvalue > 1e-3


# -------------------------------------------------------------- gradients

def test_gradients_match_central_differences(oracle_mod):
    c = synth.tiny_curve(31, 80, T=25.0, H=3)
    H, f = 3, 0.7093
    d, g_f, g_x, g_s = oracle_mod.grad(c.t, c.x, c.sigma, H, f)
    D = lambda t, x, s, ff: oracle_mod.dchi2_freqs(t, x, s, H, [ff], threads=1)[0, H - 1]  # noqa
    assert d == pytest.approx(D(c.t, c.x, c.sigma, f), rel=1e-12)
    hf = 1e-6 / 25.0
    fd_f = (D(c.t, c.x, c.sigma, f + hf) - D(c.t, c.x, c.sigma, f - hf)) / (2 * hf)
    assert g_f == pytest.approx(fd_f, rel=1e-5, abs=1e-6 * abs(d) * 25.0)
    for i in (0, 17, 41, 79):
        hx = 1e-6 * c.sigma[i]
        xp, xm = c.x.copy(), c.x.copy()
        xp[i] += hx
        xm[i] -= hx
        fd = (D(c.t, xp, c.sigma, f) - D(c.t, xm, c.sigma, f)) / (2 * hx)
        assert g_x[i] == pytest.approx(fd, rel=1e-5, abs=1e-7 * abs(d) / c.sigma[i])
        sp, sm = c.sigma.copy(), c.sigma.copy()
        sp[i] += hx
        sm[i] -= hx
        fd = (D(c.t, c.x, sp, f) - D(c.t, c.x, sm, f)) / (2 * hx)
        assert g_s[i] == pytest.approx(fd, rel=1e-5, abs=1e-7 * abs(d) / c.sigma[i])


def test_brent_refine_finds_the_peak(oracle_mod):
    c = synth.short_curve(n=400, N=4096)
    H = 3
    f0 = 1.37
    a, b = f0 - 0.004, f0 + 0.004
    fs, v = oracle_mod.refine(c.t, c.x, c.sigma, H, a, b, tol=1e-12)
    grid = np.linspace(a, b, 801)
    scan = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, H, grid)[:, H - 1]
    assert v >= scan.max() - 1e-9 * abs(v)
    assert abs(fs - grid[np.argmax(scan)]) <= (b - a) / 800
    _, g_f, _, _ = oracle_mod.grad(c.t, c.x, c.sigma, H, fs)
    _, g_far, _, _ = oracle_mod.grad(c.t, c.x, c.sigma, H, fs + 1e-5)
    assert abs(g_f) < 1e-4 * abs(g_far)


# ------------------------------------------------------------ significance

@pytest.mark.parametrize("Hp", [1, 2, 3, 5, 8, 16])
def test_chi2_survival_matches_library(oracle_mod, Hp):
    """The even-dof chi^2 survival function of p(f) (Sec. 3d) equals scipy's
    chi^2 log survival function, from the body of the distribution far into
    its tail."""
    from scipy import stats
    x = np.concatenate([[0.0, 1e-3, 0.5, 1.0], np.geomspace(2.0, 1200.0, 40)])
    got = oracle_mod.chi2_logsf_even(x, Hp)
    ref = stats.chi2.logsf(x, 2 * Hp)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    # far tail (scipy's survival function underflows): mpmath's regularised
    # upper incomplete gamma at 50 digits
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    xt = np.geomspace(2000.0, 5e6, 12)
    ref_t = [float(mpmath.log(mpmath.gammainc(Hp, a=mpmath.mpf(v) / 2, regularized=True)))
             for v in xt]
    np.testing.assert_allclose(oracle_mod.chi2_logsf_even(xt, Hp), ref_t, rtol=1e-13)
    # one harmonic: exponential distribution, ln P = -x/2
    if Hp == 1:
        np.testing.assert_allclose(got, -x / 2, rtol=1e-15, atol=0)


def test_false_alarm_is_uniform_under_the_null(oracle_mod):
    """Under a constant source, P_{2H', >= Delta chi^2}(Delta chi^2) at a fixed
    frequency is uniform on (0, 1) -- the oracle's Delta chi^2 fed through
    the oracle's survival function (Sec. 3d's reading of P)."""
    from scipy import stats
    rng = np.random.default_rng(321)
    n, R = 40, 2000
    t = np.sort(rng.uniform(0, 20, n))
    sigma = rng.uniform(0.3, 2.0, n)
    vals = np.empty((R, 2))
    for r in range(R):
        x = 1.0 + sigma * rng.standard_normal(n)
        vals[r] = oracle_mod.dchi2_freqs(t, x, sigma, 2, [0.731], threads=1)[0]
    for Hp in (1, 2):
        u = np.exp(oracle_mod.chi2_logsf_even(vals[:, Hp - 1], Hp))
        assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_false_alarm_and_adjusted_hand_values(oracle_mod):
    """fhat = f / df (at least 1) and the adjusted-Delta chi^2 factor on hand
    examples (Sec. 3d)."""
    # f_min = df: fhat = j + 1; f_min = 0: the first bin counts as one trial
    np.testing.assert_array_equal(oracle_mod.fhat(0.5, 0.5, [0, 1, 9]), [1.0, 2.0, 10.0])
    np.testing.assert_array_equal(oracle_mod.fhat(0.0, 0.25, [0, 1, 4]), [1.0, 1.0, 4.0])
    d = np.array([[0.0, 0.0], [10.0, 12.0]])
    lp = oracle_mod.log_false_alarm(d, 0.5, 0.5, [0, 3])
    np.testing.assert_allclose(lp[0], [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(lp[1, 0], math.log(4.0) - 5.0, rtol=1e-14)
    np.testing.assert_allclose(lp[1, 1], math.log(4.0) - 6.0 + math.log(7.0), rtol=1e-14)
    s = oracle_mod.adjusted_scale([100.0, 200.0], 500.0, 100)
    np.testing.assert_allclose(s, [97.0 / 400.0, 95.0 / 300.0], rtol=1e-15)


def test_adjusted_scale_is_unit_under_the_null(oracle_mod):
    """Sec. 3d's adjusted Delta chi^2 divides by the best fit's residual chi^2
    per degree of freedom.  Under a constant source with correct errors, the
    residual chi^2 of the H'-harmonic fit at a fixed frequency is chi^2 with
    n - 2H' - 1 degrees of freedom (n samples, 2H' + 1 parameters), so
    1 / s_{H'} = (chi2_0 - Delta chi^2) / (n - 2H' - 1) has mean 1 and
    variance 2 / (n - 2H' - 1).  With n = 20 a degree-of-freedom count off by
    one moves the mean by 1/15 (about 11 standard errors here), and chi2_0 in
    place of the residual by 4/15."""
    rng = np.random.default_rng(4242)
    n, R, H = 20, 4000, 2
    t = np.sort(rng.uniform(0.0, 30.0, n))
    sigma = rng.uniform(0.3, 2.0, n)
    inv = np.empty((R, H))
    for r in range(R):
        x = 3.0 + sigma * rng.standard_normal(n)
        d = oracle_mod.dchi2_freqs(t, x, sigma, H, [0.4123], threads=1)[0]
        _, _, chi0, _ = oracle_mod.moments(x, sigma)
        inv[r] = 1.0 / oracle_mod.adjusted_scale(d, chi0, n)
    for h in range(H):
        dof = n - 2 * (h + 1) - 1
        se = math.sqrt(2.0 / dof / R)
        assert abs(inv[:, h].mean() - 1.0) < 4.0 * se
        # the spread is that of chi^2_dof / dof as well
        assert abs(inv[:, h].var() - 2.0 / dof) < 0.25 * (2.0 / dof)


def test_adjusted_scale_denominator_is_the_lstsq_residual(oracle_mod):
    """The denominator chi2_0 - Delta chi^2_best is the residual chi^2 of the
    best fit: numpy's least squares on the explicit weighted design
    [1, sin 2 pi h f t, cos 2 pi h f t] at the best frequency, per H'."""
    c = synth.tiny_curve(31, 60, T=25.0, H=3, N=300, f_min=0.02, df=0.01)
    freqs = c.f_min + np.arange(c.N) * c.df
    d = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, c.H, freqs)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    best = d.max(axis=0)
    s = oracle_mod.adjusted_scale(best, chi0, c.n)
    sw = 1.0 / c.sigma
    for h in range(1, c.H + 1):
        f = freqs[np.argmax(d[:, h - 1])]
        cols = [np.ones(c.n)]
        for k in range(1, h + 1):
            cols += [np.sin(2 * np.pi * k * f * c.t), np.cos(2 * np.pi * k * f * c.t)]
        X = np.stack(cols, axis=1) * sw[:, None]
        coef, *_ = np.linalg.lstsq(X, c.x * sw, rcond=None)
        resid = float(np.sum((X @ coef - c.x * sw) ** 2))
        np.testing.assert_allclose(s[h - 1], (c.n - 2 * h - 1) / resid, rtol=1e-9)


# ------------------------------------------------------ the paper's gridding

def test_paper_grid_times_on_and_off_cell_edges(oracle_mod):
    """Times on cell edges keep their place; just below an edge they fall to
    the cell beneath (floor, Sec. 3b)."""
    df, M, T0 = 2.0 ** -10, 2 ** 12, 3.0  # dt = 1 / (M df) = 1/4
    k = np.array([0, 1, 5, 4095, 4096, 4100])
    t = T0 + k * 0.25
    tp, cells = oracle_mod.paper_grid_times(t, T0, df, M)
    np.testing.assert_array_equal(cells, k % M)
    np.testing.assert_array_equal(tp, (k % M) * 0.25)
    tb = T0 + k[1:4] * 0.25 - 1e-9
    np.testing.assert_array_equal(oracle_mod.paper_grid_times(tb, T0, df, M)[1], k[1:4] - 1)


def test_paper_gridding_is_the_fft_of_the_binned_arrays(oracle_mod):
    """The paper's Phat, Qhat (FFT of the Kronecker-delta binned weighted data
    and weights, Sec. 3b) equal the direct sums of Eq. eqPQ at the snapped
    times: numpy's FFT of explicitly binned arrays against the oracle's
    trigonometric sums."""
    rng = np.random.default_rng(17)
    n, df, M = 300, 1.0 / 512.0, 4096
    t = np.sort(rng.uniform(0.0, 400.0, n))
    T0 = t.min()
    w = rng.uniform(0.5, 2.0, n)
    c = w * rng.standard_normal(n)
    tp, cells = oracle_mod.paper_grid_times(t, T0, df, M)
    qh = np.zeros(M)
    ph = np.zeros(M)
    np.add.at(qh, cells, w)
    np.add.at(ph, cells, c)
    # sign +i (Eq. eqPQ): sum_t a[t] e^{+2 pi i m t / M} = M * ifft(a)[m]
    Q = M * np.fft.ifft(qh)
    P = M * np.fft.ifft(ph)
    m = np.arange(1, 200)
    np.testing.assert_allclose(Q[m], oracle_mod.trig_sums(tp, w, m * df), rtol=0,
                               atol=1e-9 * w.sum())
    np.testing.assert_allclose(P[m], oracle_mod.trig_sums(tp, c, m * df), rtol=0,
                               atol=1e-9 * np.abs(c).sum())


def test_paper_method_equals_least_squares_at_snapped_times(oracle_mod):
    """The host restatement of the paper's algorithm (binning, one FFT,
    identities, nested Cholesky) gives the oracle's least-squares Delta chi^2
    at the snapped times for every H' (Sec. 3b-3c)."""
    from oracle import paper_method
    c = synth.tiny_curve(21, 250, T=60.0, H=3, N=200, f_min=3 * 0.0125, df=0.0125)
    M = 4096
    bins = np.arange(c.N)
    d, times = paper_method.fchi2_paper(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins, M)
    tp, _ = oracle_mod.paper_grid_times(c.t, c.t.min(), c.df, M)
    ref, piv = oracle_mod.dchi2_bins(tp, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    strict = piv >= 1e-8
    assert strict.mean() > 0.9
    np.testing.assert_allclose(d[strict], ref[strict], rtol=0, atol=1e-9 * chi0)
    assert set(times) == {"grid_s", "fft_s", "solve_s"}


# ------------------------------------------------------------ detrending

@pytest.mark.parametrize("degree", [0, 1, 2, 3])
def test_detrend_removes_polynomials_and_is_orthogonal(oracle_mod, degree):
    """A polynomial of the fitted degree is removed exactly; in general the
    residual is weighted-orthogonal to 1, t, .., t^degree; degree 0 is the
    weighted mean of Sec. 3b."""
    rng = np.random.default_rng(degree)
    n = 400
    t = np.sort(rng.uniform(1000.0, 1600.0, n))
    sigma = rng.uniform(0.5, 2.0, n)
    w = 1.0 / sigma ** 2
    tc = (t - 1300.0) / 300.0
    poly = sum((k + 1.5) * tc ** k for k in range(degree + 1))
    r = oracle_mod.detrend(t, poly, sigma, degree)
    assert np.max(np.abs(r)) < 1e-10 * np.max(np.abs(poly))
    x = poly + np.sin(2 * np.pi * 0.37 * t) + sigma * rng.standard_normal(n)
    r = oracle_mod.detrend(t, x, sigma, degree)
    for k in range(degree + 1):
        assert abs(np.sum(w * r * tc ** k)) < 1e-9 * np.sum(w * np.abs(x) * np.abs(tc) ** k)
    if degree == 0:
        _, xbar, _, _ = oracle_mod.moments(x, sigma)
        np.testing.assert_allclose(r, x - xbar, rtol=0, atol=1e-12 * np.abs(x).max())


# ------------------------------------------- trend fitted with the harmonics

def _lstsq_resid(X, y):
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    return float(np.sum((X @ coef - y) ** 2))


@pytest.mark.parametrize("D", [1, 2, 3])
def test_joint_trend_fit_matches_lstsq(oracle_mod, D):
    """Delta chi^2 of the joint fit (Sec. 4's detrending read as a polynomial of
    degree D fitted together with the harmonics) equals the difference of two
    numpy least-squares residuals on the explicit weighted designs
    [u^0..u^D] and [u^0..u^D, sin 2 pi h f t, cos 2 pi h f t (h <= H')]."""
    c = synth.tiny_curve(40 + D, 70, T=25.0, H=3, N=40, f_min=0.07, df=0.013)
    freqs = c.f_min + np.arange(0, c.N, 7) * c.df
    d, chi0 = oracle_mod.dchi2_trend_freqs(c.t, c.x, c.sigma, c.H, D, freqs)
    sw = 1.0 / c.sigma
    u = (c.t - 0.5 * (c.t.min() + c.t.max())) / (0.5 * (c.t.max() - c.t.min()))
    P = np.vander(u, D + 1, increasing=True) * sw[:, None]
    y = c.x * sw
    r_poly = _lstsq_resid(P, y)
    np.testing.assert_allclose(chi0, r_poly, rtol=1e-10)
    for k, f in enumerate(freqs):
        for Hp in range(1, c.H + 1):
            cols = [P]
            for h in range(1, Hp + 1):
                th = 2 * np.pi * h * f * c.t
                cols.append(np.stack([np.sin(th) * sw, np.cos(th) * sw], axis=1))
            X = np.concatenate(cols, axis=1)
            np.testing.assert_allclose(d[k, Hp - 1], r_poly - _lstsq_resid(X, y),
                                       rtol=1e-8, atol=1e-9 * r_poly)


def test_joint_trend_fit_degree_zero_is_the_plain_definition(oracle_mod):
    c = synth.tiny_curve(51, 60, T=20.0, H=3, N=30, f_min=0.1, df=0.02)
    freqs = c.f_min + np.arange(c.N) * c.df
    d, chi0 = oracle_mod.dchi2_trend_freqs(c.t, c.x, c.sigma, c.H, 0, freqs)
    ref = oracle_mod.dchi2_freqs(c.t, c.x, c.sigma, c.H, freqs)
    _, _, chi0_ref, _ = oracle_mod.moments(c.x, c.sigma)
    np.testing.assert_allclose(d, ref, rtol=1e-9, atol=1e-9 * chi0_ref)
    np.testing.assert_allclose(chi0, chi0_ref, rtol=1e-12)


@pytest.mark.parametrize("D", [1, 3])
def test_joint_trend_fit_ignores_polynomials_and_bounds_subtract_first(oracle_mod, D):
    """Adding any polynomial of degree <= D in t to the data leaves the joint
    fit's Delta chi^2 unchanged; and the joint fit never falls below the
    subtract-the-trend-first reading (same baseline, more freedom)."""
    rng = np.random.default_rng(D)
    c = synth.tiny_curve(60 + D, 90, T=40.0, H=2, N=60, f_min=0.04, df=0.011)
    freqs = c.f_min + np.arange(c.N) * c.df
    d, chi0 = oracle_mod.dchi2_trend_freqs(c.t, c.x, c.sigma, c.H, D, freqs)
    tt = (c.t - c.t.mean()) / c.t.std()
    poly = sum(rng.normal(0, 3.0) * tt ** k for k in range(D + 1))
    d2, chi02 = oracle_mod.dchi2_trend_freqs(c.t, c.x + poly, c.sigma, c.H, D, freqs)
    np.testing.assert_allclose(d2, d, rtol=1e-7, atol=1e-8 * chi0)
    np.testing.assert_allclose(chi02, chi0, rtol=1e-8)
    xd = oracle_mod.detrend(c.t, c.x, c.sigma, D)
    d_first = oracle_mod.dchi2_freqs(c.t, xd, c.sigma, c.H, freqs)
    assert np.all(d >= d_first - 1e-9 * chi0)
    assert np.any(d > d_first + 1e-6 * chi0)


def test_joint_trend_fit_noiseless_signal_is_fully_explained(oracle_mod):
    """x = cubic trend + 2 harmonics of f0 (on the trial grid), no noise: at f0
    the joint fit with H' >= 2 leaves no residual, Delta chi^2 = chi^2 of the
    trend alone."""
    rng = np.random.default_rng(9)
    n, f0 = 120, 0.35
    t = np.sort(rng.uniform(0, 60.0, n))
    sigma = rng.uniform(0.5, 1.5, n)
    tt = t / 60.0
    x = 2.0 - 1.5 * tt + 0.7 * tt ** 2 + 0.4 * tt ** 3
    x += 1.2 * np.sin(2 * np.pi * f0 * t + 0.3) + 0.5 * np.cos(4 * np.pi * f0 * t - 1.1)
    d, chi0 = oracle_mod.dchi2_trend_freqs(t, x, sigma, 3, 3, [f0])
    np.testing.assert_allclose(d[0, 1:], chi0, rtol=1e-9)
    assert d[0, 0] < chi0 * (1 - 1e-3)
