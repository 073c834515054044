"""Each precision tier of the exact (ungridded) evaluation against the oracle,
on bins that include the sampling aliases of a seasonal, nightly window."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import TOL, compare, sample_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


@pytest.fixture(scope="module")
def case(oracle_mod):
    c = synth.long_curve(n=20000, N=1 << 18)
    # half-integer cycles per day: the daily and yearly window peaks make the
    # normal equations of those bins nearly singular
    centres = [int(round((0.5 * m - c.f_min) / c.df)) for m in range(1, 12)]
    centres.append(int(round((c.truth["f0"] - c.f_min) / c.df)))
    bins = sample_bins(c.N, 120, 5, windows=centres, half=3)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    return c, bins, ref, piv, chi0


# (tier, tolerance relative to chi2_0, oracle pivot below which a bin only has
# to respect the bounds).  Tier 1 (float sums) is only meant for well-posed bins.
@pytest.mark.parametrize("tier,tol,near", [(1, TOL, 1e-3), (2, 1e-6, 1e-8), (3, 1e-8, 1e-8),
                                           (4, 1e-8, 1e-8)])
def test_tier_matches_oracle(fc2, case, tier, tol, near):
    c, bins, ref, piv, chi0 = case
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        p.execute()
        got = p.exact_bins(bins, tier).T
    r = compare(got, ref, piv, chi0, tol=tol, near_alias=near)
    print(tier, r)
    assert r["ok"], (tier, r)


def test_double_float_tracks_double(fc2, case):
    """Tier 2 agrees with tier 3 far beyond the parity tolerance on every bin
    whose oracle pivot is not at a rank decision."""
    c, bins, ref, piv, chi0 = case
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        p.execute()
        d2 = p.exact_bins(bins, 2).T
        d3 = p.exact_bins(bins, 3).T
    ok = piv >= 1e-8
    err = np.abs(d2 - d3)[ok].max() / chi0
    print("tier2 vs tier3", err)
    assert err <= 1e-8


def test_fixed_point_sums_track_double_and_repeat(fc2, case):
    """Tier 4 (double-float terms, sums exact in fixed point) agrees with the
    double tier far beyond the parity tolerance wherever the oracle's pivots
    are not at a rank decision, and gives the same bits when repeated (integer
    sums do not depend on the order)."""
    c, bins, ref, piv, chi0 = case
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        p.execute()
        d3 = p.exact_bins(bins, 3).T
        d4 = p.exact_bins(bins, 4).T
        d4b = p.exact_bins(bins, 4).T
    np.testing.assert_array_equal(d4, d4b)
    ok = piv >= 1e-8
    err = np.abs(d4 - d3)[ok].max() / chi0
    print("tier4 vs tier3", err)
    assert err <= 1e-8


@pytest.mark.parametrize("last", [3, 4])
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_pipeline_on_degenerate_bins(fc2, oracle_mod, prec, last):
    """The whole pipeline (gridded solve, routing, every fix-up tier) on the
    bins that need the most precision: periods longer than the span (f near 0)
    and the daily aliases, against the oracle."""
    c = synth.long_curve(n=20000, N=1 << 18)
    one = int(round((1.0 - c.f_min) / c.df))
    bins = np.unique(np.concatenate([np.arange(0, 96), np.arange(one - 40, one + 41),
                                     np.arange(2 * one - 20, 2 * one + 21)]))
    fc2.last_tier(last)
    try:
        with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec) as p:
            d, _, _, chi0 = p.execute()
            counts = p.counts
    finally:
        fc2.last_tier(4)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0)
    print(prec, last, counts, r)
    assert r["ok"], r


def test_large_curve_full_size(fc2, oracle_mod):
    """The large single curve at full size -- about 10^6 samples at 2-min
    cadence over 4 years, H = 8, N = 2^26 trial frequencies, 2x oversampled
    grids of 2^27 points -- in mixed precision against the oracle on the
    periods longer than the span (the first bins, nearly all sent to the exact
    fix-up), a window at each signal frequency and random bins."""
    c = synth.large_curve()
    fs = [f * h for f in c.truth["fs"] for h in (1, 2)]
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        d, best, _, chi0 = p.execute()
        counts = p.counts
    bins = sample_bins(c.N, 24, 9, windows=[int(round((f - c.f_min) / c.df)) for f in fs] +
                       [int(best[-1]["j"])], half=1)
    bins = np.unique(np.concatenate([bins, np.arange(0, 2048, 64), np.arange(0, 24)]))
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0)
    print(counts, r)
    assert counts[1] > 100 and r["ok"], r


@pytest.mark.parametrize("fn", ["fc2_debug_phasor", "fc2_debug_phasor16"])
def test_double_float_phasor_accuracy(fc2, fn):
    """The exact fix-up's double-float phasors e^{2 pi i u 2^-64} (two table
    factors for the top 16 bits, or one entry of the 65536-entry table of the
    last tier, then a small rotation by the rest) against the same exact phase
    evaluated in long double: random phases over the whole 64-bit range plus
    the table and rotation boundaries, within 2^-45 absolute."""
    import ctypes
    lib = fc2.load()
    rng = np.random.default_rng(5)
    edges = [0, 1, (1 << 48) - 1, 1 << 48, (1 << 56) - 1, 1 << 56, 1 << 63, (1 << 64) - 1,
             (255 << 48) | ((1 << 48) - 1), (1 << 62) | ((1 << 48) - 1), 3 << 62]
    u = np.concatenate([np.array(edges, dtype=np.uint64),
                        rng.integers(0, 2**64, size=50000, dtype=np.uint64, endpoint=False)])
    out = np.zeros(4 * u.size, dtype=np.float32)
    rc = getattr(lib, fn)(ctypes.c_void_p(u.ctypes.data), ctypes.c_int64(u.size),
                          ctypes.c_void_p(out.ctypes.data))
    assert rc == 0
    ld = np.longdouble
    two_pi = ld("6.283185307179586476925286766559005768394338798750211641949889184615632812572")
    frac = u.astype(ld) / ld(2.0) ** 64
    frac = frac - np.round(frac)
    ref_re, ref_im = np.cos(two_pi * frac), np.sin(two_pi * frac)
    o = out.reshape(-1, 4).astype(ld)
    err = max(np.max(np.abs(o[:, 0] + o[:, 1] - ref_re)), np.max(np.abs(o[:, 2] + o[:, 3] - ref_im)))
    print(fn, "max abs error", float(err), "= 2^%.1f" % np.log2(float(err)))
    assert err <= 2.0 ** -45


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_exact_aliases_at_30_min_cadence(fc2, oracle_mod, prec):
    """The large curve's 30-minute-cadence variant (n ~ 6.7e4 over 4 years,
    H = 8): every time is a whole number of 1/48 d (up to the rounding of the
    times), so sin(2 pi h f t) vanishes on all samples wherever 2 h f / 48 is
    an integer -- f = 3 /d for h = 8, f = 6 /d for h = 4, ... -- and cosines
    equal the constant where it is even: the design matrix is rank-deficient
    there (the rank-drop rule must engage).  Those bins (on the
    trial grid: f_min = df = 24 / 2^22) with windows around them, the first
    bins and random bins, against the oracle."""
    c = synth.large_curve(cadence_min=30.0, N=1 << 22)
    # aliases f = 24 m / h that fall on a trial frequency (j + 1) df = j' 24 / 2^22
    alias_f = sorted({24.0 * m / h for h in range(1, 9) for m in range(1, 9)
                      if 24.0 * m / h <= 23.9 and (m << 22) % h == 0})
    centres = [int(round(f / c.df)) - 1 for f in alias_f]
    assert len(centres) == 7  # 3, 6, .., 21 /d
    assert all(abs((j + 1) * c.df - f) < 1e-9 for j, f in zip(centres, alias_f))
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec) as p:
        d, _, _, chi0 = p.execute()
        counts = p.counts
    bins = sample_bins(c.N, 60, 13, windows=centres, half=2)
    bins = np.unique(np.concatenate([bins, np.arange(0, 16)]))
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    # some of them are rank decisions for the oracle too (at f = 12 /d the
    # fourth and eighth cosines equal the constant on every sample; a sine
    # that vanishes is a near-zero column, which a pivot relative to the
    # column's own norm does not flag)
    at = np.searchsorted(bins, centres)
    assert np.any(piv[at, -1] < 1e-8), piv[at, -1]
    r = compare(d[:, bins].T, ref, piv, chi0)
    print(prec, counts, r)
    assert r["ok"], r
