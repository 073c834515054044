"""The paper's own gridding (Sec. 3b-3c, fc2_options.gridding = 1): weights and
weighted data binned into the lower cell of one zero-padded array, one
transform, harmonics read at multiples of the bin index, no deconvolution.
Its Delta chi^2 is the exact value for the sample times moved to their cells'
lower edges -- the oracle on those snapped times is the parity target; the
gridding error against the original times is the paper's and is not bounded."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import compare, sample_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


def paper_M(H, f_min, df, N):
    s0 = int(round(f_min / df))
    M = 1024
    while M < 4 * H * (s0 + N - 1) + 1:
        M *= 2
    return M


@pytest.mark.parametrize("prec,tol", [("mixed", 5e-6), ("fp64", 1e-10)])
def test_paper_gridding_matches_oracle_on_snapped_times(fc2, oracle_mod, prec, tol):
    c = synth.long_curve(n=3000, N=1 << 14)
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, prec,
                  gridding="paper") as p:
        d, best, _, chi0 = p.execute()
        spec = p.spectra()
        T0 = p.t0
    M = paper_M(c.H, c.f_min, c.df, c.N)
    tp, _ = oracle_mod.paper_grid_times(c.t, T0, c.df, M)
    # spectra: the direct sums of Eq. eqPQ at the snapped times
    w = 1.0 / c.sigma ** 2
    _, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    cp = w * (c.x - xbar)
    bins = sample_bins(c.N, 150, 3, windows=[0, c.N - 1, int(best[-1]["j"])])
    f = c.f_min + bins * c.df
    for g in range(3 * c.H):
        k, amp = (g + 1, w) if g < 2 * c.H else (g - 2 * c.H + 1, cp)
        ref = oracle_mod.trig_sums(tp, amp, k * f)
        err = np.max(np.abs(spec[g, bins] - ref)) / np.sum(np.abs(amp))
        assert err < tol, (prec, g, err)
    # Delta chi^2: the oracle's least squares at the snapped times
    ref, piv = oracle_mod.dchi2_bins(tp, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0)
    print(prec, r)
    assert r["ok"], (prec, r)
    # and it is the paper's gridding, not the exact periodogram: at these
    # cell widths the high harmonics carry a visible phase error
    exact = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins)
    assert np.max(np.abs(d[:, bins].T - exact)) > 1e-3 * chi0


def test_paper_gridding_with_a_wrapping_fold(fc2, oracle_mod):
    """df times the span above 1: the array wraps (exact for trial
    frequencies on the df grid); runs from different turns share cells."""
    c = synth.tiny_curve(5, 400, T=200.0, H=3, N=512, f_min=2 * 0.011, df=0.011)
    assert c.df * (c.t.max() - c.t.min()) > 1.0
    d, best, _, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed",
                                       gridding="paper")
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed",
                  gridding="paper") as p:
        T0 = p.t0
    M = paper_M(c.H, c.f_min, c.df, c.N)
    tp, _ = oracle_mod.paper_grid_times(c.t, T0, c.df, M)
    ref, piv = oracle_mod.periodogram(tp, c.x, c.sigma, c.H, c.f_min, c.df, c.N,
                                      with_pivots=True)
    r = compare(d.T, ref, piv, chi0)
    assert r["ok"], r


def test_paper_gridding_needs_an_integer_offset(fc2):
    c = synth.short_curve(n=200, N=1024)  # f_min = 0.01 is not a whole number of df steps
    with pytest.raises(fc2.Fc2Error) as e:
        fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed",
                        gridding="paper")
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG
