"""Polynomial detrending (fc2_options.detrend, Sec. 4's "detrend the data with
a polynomial fit"): the periodogram of the residuals of the weighted
least-squares polynomial, against the oracle's detrended data; and the trend
fitted together with the harmonics (fc2_options.trend_fit), against the
oracle's joint least squares."""
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


def trended_curve():
    c = synth.long_curve(n=6000, N=1 << 15)
    u = (c.t - c.t.mean()) / np.ptp(c.t)
    x = c.x + 3.0 * np.median(c.sigma) * (1.0 + 2.0 * u - 4.0 * u ** 2 + 5.0 * u ** 3)
    return c, x


@pytest.mark.parametrize("prec,degree", [("mixed", 3), ("fp64", 3), ("mixed", 1)])
def test_detrended_periodogram_matches_oracle(fc2, oracle_mod, prec, degree):
    c, x = trended_curve()
    d, best, _, chi0 = fc2.periodogram(c.t, x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample,
                                       prec, detrend=degree)
    xr = oracle_mod.detrend(c.t, x, c.sigma, degree)
    _, _, chi0_or, _ = oracle_mod.moments(xr, c.sigma)
    assert chi0 == pytest.approx(chi0_or, rel=1e-9)
    j0 = int(round((c.truth["f0"] - c.f_min) / c.df))
    bins = sample_bins(c.N, 300, 11, windows=[0, j0, int(best[-1]["j"])], half=8)
    ref, piv = oracle_mod.dchi2_bins(c.t, xr, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0_or)
    assert r["ok"], (prec, degree, r)


def test_detrend_leaves_borrowed_inputs_and_limits(fc2):
    import torch
    c, x = trended_curve()
    dev = torch.device("cuda", 0)
    td, xd, sd = (torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (c.t, x, c.sigma))
    with fc2.Plan(td, xd, sd, c.H, c.f_min, c.df, c.N, c.oversample, "mixed", detrend=2) as p:
        p.execute()
        with pytest.raises(fc2.Fc2Error) as e:
            p.backward(np.array([5]))
        assert e.value.code == fc2.FC2_ERR_UNSUPPORTED
    assert np.array_equal(xd.cpu().numpy(), x)  # the caller's data are not detrended in place
    with pytest.raises(fc2.Fc2Error) as e:
        fc2.periodogram(c.t, x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed", detrend=4)
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG


# ------------------------------------------- trend fitted with the harmonics

def _trended(c, scale=0.3):
    """The curve with a cubic trend over its span added to x."""
    tt = (c.t - 0.5 * (c.t.min() + c.t.max())) / (0.5 * (c.t.max() - c.t.min()))
    return c.x + scale * (1.0 * tt - 0.8 * tt ** 2 + 0.6 * tt ** 3)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("D", [1, 2, 3])
def test_joint_trend_fit_matches_oracle(fc2, oracle_mod, prec, D):
    """The polynomial fitted together with the harmonics (fc2_options.trend_fit)
    against the oracle's joint least squares, on random bins, the first bins
    (periods longer than the span, where trend and harmonics are nearly
    degenerate), and windows at the signal and at the GPU's best bins."""
    c = synth.short_curve()
    x = _trended(c)
    d, best, peaks, chi0 = fc2.periodogram(c.t, x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec,
                                           detrend=D, trend_fit=True)
    j0 = int(round((c.truth["f0"] - c.f_min) / c.df))
    bins = sample_bins(c.N, 400, 10 + D, windows=[j0, best[-1]["j"]], half=6)
    bins = np.unique(np.concatenate([bins, np.arange(0, 40)]))
    ref, chi0_or, piv = oracle_mod.dchi2_trend_bins(c.t, x, c.sigma, c.H, D, c.f_min, c.df,
                                                    bins, with_pivots=True)
    assert chi0 == pytest.approx(chi0_or, rel=1e-9)
    r = compare(d[:, bins].T, ref, piv, chi0_or)
    assert r["ok"], r
    for h in range(c.H):
        jb = best[h]["j"]
        assert jb in set(bins.tolist())
        k = int(np.searchsorted(bins, jb))
        # the record's value comes from exact sums at its bin
        assert best[h]["dchi2"] == pytest.approx(ref[k, h], abs=1e-7 * chi0_or)
        assert best[h]["dchi2"] >= ref[:, h].max() - TOL * chi0_or
    assert abs(best[-1]["f"] - c.truth["f0"]) < 2 * c.df


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_joint_trend_fit_ignores_added_polynomials(fc2, prec):
    """Adding a polynomial of degree <= D to the data changes nothing beyond
    the parity tolerance: the trend is part of every model."""
    c = synth.short_curve(n=600, N=4096)
    D = 2
    d1, _, _, chi1 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec,
                                     detrend=D, trend_fit=True)
    tt = c.t / 100.0
    d2, _, _, chi2 = fc2.periodogram(c.t, c.x + 3.0 - 2.0 * tt + 1.5 * tt ** 2, c.sigma, c.H,
                                     c.f_min, c.df, c.N, 2, prec, detrend=D, trend_fit=True)
    assert chi2 == pytest.approx(chi1, rel=1e-7)
    assert np.max(np.abs(d2 - d1)) <= TOL * chi1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_joint_trend_fit_long_curve_scaled(fc2, oracle_mod, prec):
    """Seasonal/nightly sampling over 3000 d with a trend, 4x oversampled grids
    (unpacked transforms in both precisions), D = 3, H = 6."""
    c = synth.long_curve(n=8000, N=1 << 16)
    x = _trended(c, scale=0.05)
    d, best, _, chi0 = fc2.periodogram(c.t, x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample,
                                       prec, detrend=3, trend_fit=True)
    j0 = int(round((c.truth["f0"] - c.f_min) / c.df))
    one = int(round((1.0 - c.f_min) / c.df))
    bins = sample_bins(c.N, 200, 33, windows=[j0, one, best[-1]["j"]], half=4)
    bins = np.unique(np.concatenate([bins, np.arange(0, 24)]))
    ref, chi0_or, piv = oracle_mod.dchi2_trend_bins(c.t, x, c.sigma, c.H, 3, c.f_min, c.df, bins,
                                                    with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0_or)
    assert r["ok"], r


def test_joint_trend_fit_options(fc2):
    c = synth.short_curve(n=300, N=2048)
    with pytest.raises(fc2.Fc2Error) as e:   # trend_fit needs a degree
        fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed", trend_fit=True)
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed", detrend=1,
                  trend_fit=True) as p:
        p.execute()
        with pytest.raises(fc2.Fc2Error) as e:
            p.backward([10])
        assert e.value.code == fc2.FC2_ERR_UNSUPPORTED
