"""Polynomial detrending (fc2_options.detrend, Sec. 4's "detrend the data with
a polynomial fit"): the periodogram of the residuals of the weighted
least-squares polynomial, against the oracle's detrended data."""
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
