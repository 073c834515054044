"""Significance of the trial frequencies (Sec. 3d) through the C ABI: ln p(f)
for every bin and H', its minimum per H', and the adjusted-Delta chi^2 factor,
against the oracle's formulas applied to the library's own Delta chi^2."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_significance_matches_oracle_formula(fc2, oracle_mod, prec):
    import torch
    c = synth.short_curve()
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec) as p:
        with pytest.raises(fc2.Fc2Error) as e:
            p.significance()  # no execute yet
        assert e.value.code == fc2.FC2_ERR_INVALID_ARG
        d, best, _, chi0 = p.execute()
        lp, jmin, lpmin, adj = p.significance(log_p=True)
        dev = torch.empty((c.H, c.N), dtype=torch.float64, device="cuda")
        _, jmin2, lpmin2, _ = p.significance(log_p=dev)
    ref = oracle_mod.log_false_alarm(d.T, c.f_min, c.df, np.arange(c.N)).T  # [H, N]
    np.testing.assert_allclose(lp, ref, rtol=1e-12, atol=1e-3)
    assert np.array_equal(dev.cpu().numpy(), lp)
    assert np.array_equal(jmin, jmin2) and np.array_equal(lpmin, lpmin2)
    for h in range(c.H):
        jr = int(np.argmin(ref[h]))
        assert jmin[h] == jr or ref[h, jmin[h]] - ref[h, jr] <= 2e-3, (h, jmin[h], jr)
        assert lpmin[h] == pytest.approx(ref[h, jmin[h]], abs=1e-3)
    np.testing.assert_allclose(adj, oracle_mod.adjusted_scale([b["dchi2"] for b in best],
                                                              chi0, c.n), rtol=1e-12)
    # the injected 1.37 /d signal is the most significant frequency at H' = 3
    assert abs(c.f_min + jmin[2] * c.df - 1.37) < 3 * c.df


def test_significance_on_the_long_curve_sample(fc2, oracle_mod):
    """Scaled long-curve workload (seasonal, nightly): ln p on sampled bins from
    the oracle's own Delta chi^2 agrees to the Delta chi^2 tolerance."""
    from tests.parity import NEAR_ALIAS, TOL, sample_bins
    c = synth.long_curve(n=8000, N=1 << 16)
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        d, best, _, chi0 = p.execute()
        lp, jmin, lpmin, adj = p.significance(log_p=True)
    bins = sample_bins(c.N, 400, 9, windows=[int(jmin[-1]), int(best[-1]["j"])])
    dor, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    ref = oracle_mod.log_false_alarm(dor, c.f_min, c.df, bins).T
    strict = (piv >= NEAR_ALIAS).T  # Delta chi^2 itself is only bounded elsewhere
    # ln p moves by -1/2 per unit of Delta chi^2 (plus a bounded log term)
    assert np.max(np.abs(lp[:, bins] - ref)[strict]) <= 0.5 * TOL * chi0 + 1e-2
