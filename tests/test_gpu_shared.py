"""Shared sampling in batches (fc2_options.shared_sampling): many sources at
the same epochs with proportional errors share the weights' transforms.
Results equal those of independent curves and the oracle."""
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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_shared_sampling_matches_independent_curves_and_oracle(fc2, oracle_mod, prec):
    b = synth.shared_field(C=12, n=600, N=1 << 13)
    ind, pk_i, _ = fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N,
                                       2, prec, top_k=4)
    shr, pk_s, st = fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N,
                                        2, prec, top_k=4, shared_sampling=True)
    pos = 0
    for c in range(b.C):
        cur = b.curve(c)
        blk = slice(pos, pos + cur.H * cur.N)
        pos += cur.H * cur.N
        _, _, chi0, _ = oracle_mod.moments(cur.x, cur.sigma)
        assert np.max(np.abs(shr[blk] - ind[blk])) <= 2e-5 * chi0, c
        for a, bb in zip(pk_s[c], pk_i[c]):
            assert a["j"] == bb["j"] or abs(a["dchi2"] - bb["dchi2"]) <= 1e-4 * chi0
        if c % 3:
            continue
        block = shr[blk].reshape(cur.H, cur.N)
        bins = sample_bins(cur.N, 100, c, windows=[int(pk_s[c][0]["j"]), 0], half=4)
        ref, piv = oracle_mod.dchi2_bins(cur.t, cur.x, cur.sigma, cur.H, cur.f_min, cur.df, bins,
                                         with_pivots=True)
        r = compare(block[:, bins].T.astype(np.float64), ref, piv, chi0)
        assert r["ok"], (c, prec, r)
    assert st["graphs"] >= 1


def test_shared_sampling_rejects_different_epochs(fc2):
    b = synth.shared_field(C=4, n=300, N=1 << 12)
    t = b.t.copy()
    t[b.offsets[2] + 7] += 1e-3  # curve 2 has one different epoch
    with pytest.raises(fc2.Fc2Error) as e:
        fc2.execute_batched(b.offsets, t, b.x, b.sigma, b.H, b.f_min, b.df, b.N, 2, "mixed",
                            shared_sampling=True)
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG
    s = b.sigma.copy()
    s[b.offsets[1] + 3] *= 1.5  # errors no longer proportional
    with pytest.raises(fc2.Fc2Error) as e:
        fc2.execute_batched(b.offsets, b.t, b.x, s, b.H, b.f_min, b.df, b.N, 2, "mixed",
                            shared_sampling=True)
    assert e.value.code == fc2.FC2_ERR_INVALID_ARG
