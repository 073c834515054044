"""The two spreading kernels: tiles of one sample set whose samples fit one
staging batch are summed cell by cell by the single-batch kernel, the others
(and, when forced, every tile) by the general kernel.  Both sum each cell's
samples in sorted order with the same arithmetic, so the spectra and the
periodograms agree bit for bit."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import compare, sample_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    yield _fc2
    _fc2.spread_force_general(False)


def _spectra(fc2, c, prec, general):
    fc2.spread_force_general(general)
    try:
        with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec) as p:
            d = p.execute()[0]
            return p.spectra(), d
    finally:
        fc2.spread_force_general(False)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("logN", [12, 16])
def test_single_batch_spread_equals_general_single(fc2, oracle_mod, prec, logN):
    """A short curve on unpacked grids: on 2^12 trial frequencies the higher
    harmonic multiples wrap around their grids (keys shifted by the grid
    length), on 2^16 none does; spread both ways."""
    c = synth.short_curve(n=700, N=1 << logN)
    s_own, d_own = _spectra(fc2, c, prec, False)
    s_tile, d_tile = _spectra(fc2, c, prec, True)
    assert np.array_equal(s_own, s_tile)
    assert np.array_equal(d_own, d_tile)
    # and the spectra are the direct sums of Eq. eqPQ
    w = 1.0 / c.sigma ** 2
    W, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    bins = sample_bins(c.N, 100, 4, windows=[0, c.N - 1])
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec) as p:
        t0 = p.t0
    f = c.f_min + bins * c.df
    tol = 1e-10 if prec == "fp64" else 2e-6
    for g in range(3 * c.H):
        k, amp = (g + 1, w) if g < 2 * c.H else (g - 2 * c.H + 1, w * (c.x - xbar))
        ref = oracle_mod.trig_sums(c.t - t0, amp, k * f)
        err = np.max(np.abs(s_own[g, bins] - ref)) / np.sum(np.abs(amp))
        assert err < tol, (prec, g, err)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_single_batch_spread_equals_general_batched(fc2, oracle_mod, prec):
    """A small survey batch with a few dense curves (tiles beyond one staging
    batch go to the general kernel): the batched periodograms and peak records
    with every tile in the general kernel are identical, and match the
    oracle."""
    b = synth.survey_batch(seed=5, C=16, N=1 << 13, n_median=2000.0, n_hi=20000)
    outs = []
    for general in (False, True):
        fc2.spread_force_general(general)
        try:
            out, peaks, _ = fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min,
                                                b.df, b.N, 2, prec, autotune="fixed")
        finally:
            fc2.spread_force_general(False)
        outs.append((out, peaks))
    assert np.array_equal(outs[0][0], outs[1][0])
    ra, rz = outs[0][1].records, outs[1][1].records
    for name in ("j", "dchi2", "H", "A"):
        assert np.array_equal(ra[name], rz[name]), name
    out = outs[0][0]
    pos = 0
    for c in range(b.C):
        cur = b.curve(c)
        block = out[pos:pos + cur.H * cur.N].reshape(cur.H, cur.N)
        pos += cur.H * cur.N
        if c % 5:
            continue
        bins = sample_bins(cur.N, 120, c, windows=[int(np.argmax(block[-1]))], half=6)
        ref, piv = oracle_mod.dchi2_bins(cur.t, cur.x, cur.sigma, cur.H, cur.f_min, cur.df, bins,
                                         with_pivots=True)
        _, _, chi0, _ = oracle_mod.moments(cur.x, cur.sigma)
        r = compare(block[:, bins].T.astype(np.float64), ref, piv, chi0)
        assert r["ok"], (c, r)
