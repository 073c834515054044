"""Seeded random configurations through the C ABI against the oracle: H,
N, trial grid (integer and fractional offsets), oversampling, precision, the
paper's gridding, detrending and unsorted input, on sampled bins of small
curves (tolerances and near-alias rules of tests/parity.py)."""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import compare, sample_bins

pytestmark = pytest.mark.gpu

CASES = list(range(64))


@pytest.fixture(scope="module")
def fc2():
    from paper_0901_1913_gb300 import _fc2
    _fc2.load()
    return _fc2


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(60, 1500))
    T = float(rng.uniform(5.0, 400.0))
    H = int(rng.integers(1, 9))
    N = int(rng.choice([257, 1000, 2048, 4093, 8192]))
    df = float(rng.uniform(0.2, 1.5)) / T
    integer_offset = bool(rng.integers(0, 2))
    f_min = float(rng.integers(0, 5)) * df if integer_offset else float(rng.uniform(0.0, 0.3))
    c = synth.tiny_curve(seed, n, T=T, H=H, N=N, f_min=f_min, df=df,
                         signal=float(rng.uniform(0.0, 3.0)))
    opts = dict(prec=str(rng.choice(["mixed", "fp64"])), oversample=int(rng.choice([2, 4])),
                gridding="paper" if (integer_offset and rng.uniform() < 0.3) else "kernel",
                detrend=int(rng.choice([0, 0, 1, 3])), shuffle=bool(rng.integers(0, 2)))
    return c, opts


@pytest.mark.parametrize("seed", CASES)
def test_random_configuration_matches_oracle(fc2, oracle_mod, seed):
    c, o = draw(seed)
    t, x, s = c.t, c.x, c.sigma
    if o["shuffle"]:
        p = np.random.default_rng(seed).permutation(c.n)
        t, x, s = t[p], x[p], s[p]
    with fc2.Plan(t, x, s, c.H, c.f_min, c.df, c.N, o["oversample"], o["prec"],
                  gridding=o["gridding"], detrend=o["detrend"]) as plan:
        d, best, peaks, chi0 = plan.execute()
        T0 = plan.t0
    xr = oracle_mod.detrend(c.t, c.x, c.sigma, o["detrend"]) if o["detrend"] else c.x
    tt = c.t
    if o["gridding"] == "paper":
        s0 = int(round(c.f_min / c.df))
        M = 1024
        while M < 4 * c.H * (s0 + c.N - 1) + 1:
            M *= 2
        tt, _ = oracle_mod.paper_grid_times(c.t, T0, c.df, M)
    bins = sample_bins(c.N, 60, seed, windows=[0, c.N - 1, int(best[-1]["j"])], half=3)
    ref, piv = oracle_mod.dchi2_bins(tt, xr, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    _, _, chi0_or, _ = oracle_mod.moments(xr, c.sigma)
    assert chi0 == pytest.approx(chi0_or, rel=1e-9)
    r = compare(d[:, bins].T, ref, piv, chi0_or)
    assert r["ok"], (seed, o, c.n, c.H, c.N, r)


@pytest.mark.parametrize("seed", list(range(12)))
def test_random_batch_matches_oracle(fc2, oracle_mod, seed):
    """Random batches: uneven n and H, two trial-grid lengths (two chunks),
    both precisions; or, every third seed, a shared-sampling field."""
    rng = np.random.default_rng(5000 + seed)
    prec = "fp64" if seed % 4 == 3 else "mixed"
    if seed % 3 == 2:
        b = synth.shared_field(seed=seed, C=int(rng.integers(3, 9)), n=int(rng.integers(100, 800)),
                               N=int(rng.choice([1 << 11, 1 << 12])), H=int(rng.integers(1, 7)))
        kw = dict(shared_sampling=True)
    else:
        C = int(rng.integers(3, 9))
        curves = [synth.tiny_curve(100 * seed + c, int(rng.integers(40, 900)),
                                   T=float(rng.uniform(20, 500)), H=int(rng.integers(1, 9)),
                                   N=int(rng.choice([1500, 4096])), f_min=0.0, df=1.0)
                  for c in range(C)]
        for cur in curves:  # trial grid from the span: about 1/T spacing to 10 /d
            cur.df = 0.8 / float(np.ptp(cur.t))
            cur.f_min = float(rng.integers(0, 3)) * cur.df
        offsets = np.concatenate([[0], np.cumsum([cur.n for cur in curves])]).astype(np.int64)
        b = synth.Batch(offsets, np.concatenate([cu.t for cu in curves]),
                        np.concatenate([cu.x for cu in curves]),
                        np.concatenate([cu.sigma for cu in curves]),
                        np.array([cu.H for cu in curves], dtype=np.int32),
                        np.array([cu.f_min for cu in curves]), np.array([cu.df for cu in curves]),
                        np.array([cu.N for cu in curves], dtype=np.int64), 2, [{}] * C)
        kw = {}
    out, peaks, _ = fc2.execute_batched(b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N, 2,
                                        prec, top_k=4, **kw)
    pos = 0
    for c in range(b.C):
        cur = b.curve(c)
        blk = out[pos:pos + cur.H * cur.N].reshape(cur.H, cur.N)
        pos += cur.H * cur.N
        bins = sample_bins(cur.N, 40, seed + c, windows=[0, cur.N - 1], half=2)
        ref, piv = oracle_mod.dchi2_bins(cur.t, cur.x, cur.sigma, cur.H, cur.f_min, cur.df, bins,
                                         with_pivots=True)
        _, _, chi0, _ = oracle_mod.moments(cur.x, cur.sigma)
        r = compare(blk[:, bins].T.astype(np.float64), ref, piv, chi0)
        assert r["ok"], (seed, c, prec, kw, r)
    assert pos == out.size
