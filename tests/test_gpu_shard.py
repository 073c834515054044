"""Band sharding of one curve, with the bands run one after another on one
GPU: every band matches the oracle on its own bins, and the merged records
match the unsharded run and the oracle."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import shard, synth
from tests.parity import TOL, argmax_ok, compare, sample_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


@pytest.mark.parametrize("world", [2, 3])
def test_bands_match_unsharded(fc2, oracle_mod, world):
    c = synth.long_curve(n=20000, N=1 << 16)
    K = 8
    with fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed",
                  top_k=K) as p:
        d_full, best_full, peaks_full, chi0 = p.execute()
    recs, parts = [], []
    for band in shard.band_partition(c.N, world):
        fm, nb = shard.band_curve_args(c.f_min, c.df, band)
        with fc2.Plan(c.t, c.x, c.sigma, c.H, fm, c.df, nb, c.oversample, "mixed",
                      top_k=K + 2) as p:
            d, best, peaks, _ = p.execute()
        recs.append(shard.band_record(band, best, peaks, (d[-1, 0], d[-1, -1])))
        parts.append(d)
    d_cat = np.concatenate(parts, axis=1)
    best, peaks = shard.merge_records(recs, K)
    # every band against the oracle at the parity tolerance: random bins, both
    # band edges, and windows at the merged and unsharded best bins
    edges = [b for band in shard.band_partition(c.N, world) for b in (band[0], band[1] - 1)]
    centres = edges + [r["j"] for r in best] + [r["j"] for r in best_full]
    bins = sample_bins(c.N, 200, 17, windows=centres, half=2)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d_cat[:, bins].T, ref, piv, chi0)
    assert r["ok"], r
    r = compare(d_full[:, bins].T, ref, piv, chi0)
    assert r["ok"], r
    for h in range(c.H):
        j1, j2 = best[h]["j"], best_full[h]["j"]
        assert argmax_ok(j1, j2, ref[:, h], chi0, bins)
    full_j = [q["j"] for q in peaks_full]
    for q, r in zip(peaks, peaks_full):
        assert q["j"] in full_j or abs(q["dchi2"] - r["dchi2"]) <= TOL * chi0
