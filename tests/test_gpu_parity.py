"""Parity of the CUDA path (through the C ABI) with the CPU oracle."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import TOL, argmax_ok, compare, sample_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 2e-6)])
def test_spectra_match_direct_sums(fc2, oracle_mod, prec, tol):
    """P(k f_j), Q(k f_j) from spread + FFT + deconvolution equal the direct
    sums of Eq. eqPQ (relative to sum |c_i|)."""
    c = synth.short_curve(n=700, N=4096)
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec) as p:
        p.execute()
        spec = p.spectra()
        t0 = p.t0
    w = 1.0 / c.sigma ** 2
    W, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    cp = w * (c.x - xbar)
    bins = sample_bins(c.N, 200, 1, windows=[0, c.N - 1])
    f = c.f_min + bins * c.df
    H = c.H
    for g in range(3 * H):
        k, amp = (g + 1, w) if g < 2 * H else (g - 2 * H + 1, cp)
        ref = oracle_mod.trig_sums(c.t - t0, amp, k * f)
        err = np.max(np.abs(spec[g, bins] - ref)) / np.sum(np.abs(amp))
        assert err < tol, (prec, g, err)


def test_packed_spectra_match_direct_sums(fc2, oracle_mod):
    """With f_min a whole number of df steps and 4x grids, the mixed path packs
    Q_k + i P_k into one transform; the unpacked spectra still equal the direct
    sums of Eq. eqPQ."""
    c = synth.long_curve(n=3000, N=1 << 14)
    assert abs(c.f_min / c.df - round(c.f_min / c.df)) < 1e-12 and c.oversample == 4
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed") as p:
        p.execute()
        spec = p.spectra()
        t0 = p.t0
    w = 1.0 / c.sigma ** 2
    W, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    cp = w * (c.x - xbar)
    bins = sample_bins(c.N, 200, 2, windows=[0, c.N - 1])
    f = c.f_min + bins * c.df
    for g in range(3 * c.H):
        k, amp = (g + 1, w) if g < 2 * c.H else (g - 2 * c.H + 1, cp)
        ref = oracle_mod.trig_sums(c.t - t0, amp, k * f)
        err = np.max(np.abs(spec[g, bins] - ref)) / np.sum(np.abs(amp))
        assert err < 2e-6, (g, err)


@pytest.mark.parametrize("fft_kernel,fft_group", [("r64", 0), ("r16", 0), ("bulk", 0),
                                                  ("r32", 0), ("r32x", 0), ("r64", 1),
                                                  ("bulk", 2)])
@pytest.mark.parametrize("logN,oversample", [(14, 4), (19, 4), (22, 4), (19, 2), (18, 2)])
def test_fft_kernel_families_match_direct_sums(fc2, oracle_mod, fft_kernel, fft_group, logN,
                                               oversample):
    """Every float transform kernel family, on pass plans (8, 8), (11, 10) and
    (12, 12) with packed grids and (10, 10) and (10, 9) with unpacked ones,
    gives spectra equal to the direct sums of Eq. eqPQ."""
    c = synth.long_curve(n=3000, N=1 << logN)
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, oversample, "mixed",
                  fft_kernel=fft_kernel, fft_group=fft_group) as p:
        p.execute()
        spec = p.spectra()
        t0 = p.t0
    w = 1.0 / c.sigma ** 2
    W, xbar, _, _ = oracle_mod.moments(c.x, c.sigma)
    cp = w * (c.x - xbar)
    bins = sample_bins(c.N, 120, logN, windows=[0, c.N // 2, c.N - 1])
    f = c.f_min + bins * c.df
    # float transform roundoff grows with the length: ~log2(M) * 2^-24 relative
    tol = 2e-6 if logN < 20 else 1e-5
    errs = []
    for g in range(3 * c.H):
        k, amp = (g + 1, w) if g < 2 * c.H else (g - 2 * c.H + 1, cp)
        ref = oracle_mod.trig_sums(c.t - t0, amp, k * f)
        errs.append(np.max(np.abs(spec[g, bins] - ref)) / np.sum(np.abs(amp)))
    print(fft_kernel, logN, oversample, max(errs))
    assert max(errs) < tol, (fft_kernel, logN, oversample, int(np.argmax(errs)), max(errs))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_short_curve_full_periodogram(fc2, oracle_mod, prec):
    c = synth.short_curve()
    d, best, peaks, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec)
    ref, piv = oracle_mod.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, with_pivots=True)
    _, _, chi0_or, _ = oracle_mod.moments(c.x, c.sigma)
    assert chi0 == pytest.approx(chi0_or, rel=1e-12)
    r = compare(d.T, ref, piv, chi0_or)
    assert r["ok"], r
    for h in range(c.H):
        jo = int(np.argmax(ref[:, h]))
        assert argmax_ok(best[h]["j"], jo, ref[:, h], chi0_or), (h, best[h]["j"], jo)
        # the record's value and coefficients come from direct sums at its bin
        assert best[h]["dchi2"] == pytest.approx(ref[best[h]["j"], h], abs=1e-7 * chi0_or)
        A, _ = oracle_mod.coeffs(c.t, c.x, c.sigma, h + 1, c.f_min + best[h]["j"] * c.df)
        np.testing.assert_allclose(best[h]["A"], A, atol=1e-6 * np.abs(A).max())
    # true frequency 1.37 /d is the H = 3 winner
    assert abs(best[2]["f"] - 1.37) < 2 * c.df


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_peaks_are_oracle_local_maxima(fc2, oracle_mod, prec):
    """The top-K peak records against the oracle's full periodogram: each
    record's bin is a local maximum of the oracle's Delta chi^2_H up to the
    parity tolerance, its value is the oracle's, the list is in decreasing
    order, and the oracle's K largest local maxima are the records' bins up to
    near-ties (values within the tolerance)."""
    c = synth.short_curve()
    d, best, peaks, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec)
    ref = oracle_mod.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N)
    row = ref[:, c.H - 1]
    tol = TOL * chi0
    js = [p["j"] for p in peaks]
    assert js[0] == best[c.H - 1]["j"]
    vals = [p["dchi2"] for p in peaks]
    assert all(vals[i] >= vals[i + 1] for i in range(len(vals) - 1))
    for p in peaks:
        j = p["j"]
        assert abs(p["dchi2"] - row[j]) <= tol
        assert j == 0 or row[j] >= row[j - 1] - tol
        assert j == c.N - 1 or row[j] >= row[j + 1] - tol
    lm = [(row[j], j) for j in range(c.N)
          if (j == 0 or row[j] > row[j - 1]) and (j == c.N - 1 or row[j] >= row[j + 1])]
    lm.sort(key=lambda v: (-v[0], v[1]))
    for (v_or, j_or), p in zip(lm[:len(js)], peaks):
        assert j_or == p["j"] or abs(v_or - row[p["j"]]) <= tol


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_long_curve_scaled(fc2, oracle_mod, prec):
    """Seasonal/nightly sampling of the long-curve workload, scaled to 8000
    samples and 2^16 bins, 4x oversampled grids."""
    c = synth.long_curve(n=8000, N=1 << 16, T=3000.0)
    d, best, peaks, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N,
                                           c.oversample, prec)
    f0 = c.truth["f0"]
    jf0 = int(round((f0 - c.f_min) / c.df))
    bins = sample_bins(c.N, 1500, 5, windows=[jf0, 2 * jf0, jf0 // 2, best[-1]["j"],
                                               int(round((1.0 - c.f_min) / c.df))])
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0)
    assert r["ok"], r


def test_wrapping_fold(fc2, oracle_mod):
    """k df (t_max - t_min) > 1: samples wrap the fold period, exercising the
    key sort and the periodic spreading."""
    c = synth.tiny_curve(3, 300, T=200.0, H=3, N=512, f_min=0.02, df=0.011)
    for prec in ("fp64", "mixed"):
        d, best, peaks, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, prec)
        ref, piv = oracle_mod.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N,
                                          with_pivots=True)
        r = compare(d.T, ref, piv, chi0)
        assert r["ok"], (prec, r)


def test_unsorted_input_and_determinism(fc2):
    c = synth.short_curve(n=500, N=2048)
    p = np.random.default_rng(0).permutation(c.n)
    a = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed")[0]
    b = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed")[0]
    u = fc2.periodogram(c.t[p], c.x[p], c.sigma[p], c.H, c.f_min, c.df, c.N, 2, "mixed")[0]
    assert np.array_equal(a, b)  # bitwise reproducible
    np.testing.assert_allclose(u, a, rtol=0, atol=1e-6 * a.max())


def test_device_side_validation(fc2):
    c = synth.short_curve(n=64, N=256)
    s = c.sigma.copy()
    s[5] = 0.0
    with pytest.raises(fc2.Fc2Error) as e:
        fc2.periodogram(c.t, c.x, s, c.H, c.f_min, c.df, c.N)
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG
    x = c.x.copy()
    x[3] = np.nan
    with pytest.raises(fc2.Fc2Error):
        fc2.periodogram(c.t, x, c.sigma, c.H, c.f_min, c.df, c.N)


@pytest.mark.parametrize("prec,N,os_", [("fp64", 1 << 21, 4), ("mixed", 1 << 23, 4)])
def test_three_pass_transform(fc2, oracle_mod, prec, N, os_):
    """Grids long enough for three FFT passes (the middle pass writes the
    blocked layout of a non-final pass); sampled bins against the oracle."""
    c = synth.long_curve(n=3000, N=N, T=3000.0)
    d, best, peaks, chi0 = fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, os_, prec)
    jf0 = int(round((c.truth["f0"] - c.f_min) / c.df))
    bins = sample_bins(c.N, 300, 9, windows=[jf0, best[-1]["j"], c.N - 1], half=16)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins, with_pivots=True)
    r = compare(d[:, bins].T, ref, piv, chi0)
    assert r["ok"], r


def test_autotuned_plan_matches_fixed_plan(fc2, oracle_mod):
    """The autotuner only changes the transform's pass plan and kernel family:
    results agree with the fixed plan up to float rounding."""
    c = synth.long_curve(n=20000, N=1 << 18)
    out = []
    for tune in (False, True, True):  # the second tuned plan reuses the cached choice
        with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed",
                      autotune=tune) as p:
            d, best, _, chi0 = p.execute()
        out.append((d, best, chi0))
    for d, best, chi0 in out[1:]:
        assert np.max(np.abs(d - out[0][0])) <= 2e-5 * chi0
        assert best[-1]["j"] == out[0][1][-1]["j"]
    assert np.array_equal(out[1][0], out[2][0])
    # the tuned plan's results against the oracle at the parity tolerance
    bins = sample_bins(c.N, 200, 21, windows=[out[1][1][-1]["j"]], half=4)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(out[1][0][:, bins].T, ref, piv, out[1][2])
    assert r["ok"], r


def test_pool_reuse_and_trim(fc2):
    """Plans created one after another reuse the library's device pool and give
    identical results; trimming the pool between plans changes nothing."""
    c = synth.short_curve(n=500, N=4096)
    outs = []
    for it in range(3):
        with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed") as p:
            outs.append(p.execute()[0])
        if it == 1:
            fc2.trim_device_memory(0)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
