"""fc2_dchi2_exact_noalloc: the allocation-free exact evaluation.

For callers that cannot allocate device memory when they need an answer (their
memory is reserved by another allocator, or an allocation's implicit
synchronisation is not acceptable), this entry point keeps its intermediates
in a fixed-size device array owned by the library.  It must give the exact
Delta chi^2 of the least-squares definition (the CPU oracle), call after call,
over every code path of the fixed scratch layout: one and several moment
blocks (n above 8192), one and several sample chunks per bin (n above
131,072), the harmonic capacities 1..4 and 8 (H = 5..8 pad to 8), the full 128
bins, and the device-side rejection of sigma <= 0 followed by a valid call.

Collected last (file name), so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import TOL, compare, sample_bins

pytestmark = pytest.mark.gpu


def _entry():
    from paper_0901_1913_gb300 import _fc2
    lib = _fc2.load()
    fn = lib.fc2_dchi2_exact_noalloc
    fn.argtypes = [ctypes.c_void_p] * 3 + [
        ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def _call(fn, dev_arrays, n, H, f_min, df, bins_dev, nb, out, stream):
    t, x, s = dev_arrays
    return fn(t.data_ptr(), x.data_ptr(), s.data_ptr(), n, H, f_min, df, bins_dev.data_ptr(), nb,
              out.data_ptr(), stream)


def _curve(case):
    if case == "short":
        c = synth.short_curve()                  # n = 1000: one block, one chunk, H = 3
        return c, c.H, 128
    if case == "long_h5":
        c = synth.long_curve(n=300_000, N=1 << 20)   # 37 moment blocks, 64 chunks
        return c, 5, 128
    c = synth.long_curve(n=20_000, N=1 << 18)        # 3 blocks, 10 chunks, H = 8
    return c, 8, 128


@pytest.mark.parametrize("case", ["short", "long_h5", "long_h8"])
def test_noalloc_matches_oracle_twice(case, oracle_mod):
    import torch

    from paper_0901_1913_gb300 import _fc2
    fn = _entry()
    c, H, nb = _curve(case)
    f0 = c.truth.get("f0", 1.0)
    centres = [int(round((f0 - c.f_min) / c.df)), 0, int(round((1.0 - c.f_min) / c.df))]
    bins = sample_bins(c.N, nb, 4, windows=centres, half=2)
    rng = np.random.default_rng(5)
    bins = np.sort(rng.choice(bins, size=nb, replace=False))
    assert bins.size == nb
    dev = torch.device("cuda", 0)
    arrs = tuple(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (c.t, c.x, c.sigma))
    b = torch.from_numpy(bins.astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full((H, nb), float("nan"), dtype=torch.float64, device=dev)
        rc = _call(fn, arrs, c.n, H, c.f_min, c.df, b, nb, out, stream)
        assert rc == 0, _fc2.status_string(rc)
        outs.append(out.cpu().numpy())
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, H, c.f_min, c.df, bins, with_pivots=True)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    for o in outs:
        r = compare(o.T, ref, piv, chi0)
        assert r["ok"], r
        assert r["n_strict"] > 0
    np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_limits_and_invalid_sigma(oracle_mod):
    import torch

    from paper_0901_1913_gb300 import _fc2
    fn = _entry()
    c = synth.short_curve()
    dev = torch.device("cuda", 0)
    bins = np.arange(0, c.N, c.N // 64, dtype=np.int64)[:64]
    b = torch.from_numpy(bins).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    arrs = tuple(torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (c.t, c.x, c.sigma))
    out = torch.zeros((c.H, 129), dtype=torch.float64, device=dev)
    # sizes beyond the fixed scratch are refused before anything runs
    assert _call(fn, arrs, c.n, c.H, c.f_min, c.df, b, 129, out, stream) == _fc2.FC2_ERR_INVALID_ARG
    assert _call(fn, arrs, c.n, 9, c.f_min, c.df, b, 64, out, stream) == _fc2.FC2_ERR_INVALID_ARG
    assert _call(fn, arrs, (1 << 22) + 1, c.H, c.f_min, c.df, b, 64, out,
                 stream) == _fc2.FC2_ERR_INVALID_ARG
    # one sigma <= 0: rejected on the device; the next valid call is unaffected
    bad = c.sigma.copy()
    bad[123] = 0.0
    bad_arrs = (arrs[0], arrs[1], torch.from_numpy(bad).to(dev))
    out = torch.zeros((c.H, 64), dtype=torch.float64, device=dev)
    assert _call(fn, bad_arrs, c.n, c.H, c.f_min, c.df, b, 64, out,
                 stream) == _fc2.FC2_ERR_INVALID_ARG
    bad[123] = -0.05
    bad_arrs = (arrs[0], arrs[1], torch.from_numpy(bad).to(dev))
    assert _call(fn, bad_arrs, c.n, c.H, c.f_min, c.df, b, 64, out,
                 stream) == _fc2.FC2_ERR_INVALID_ARG
    rc = _call(fn, arrs, c.n, c.H, c.f_min, c.df, b, 64, out, stream)
    assert rc == 0, _fc2.status_string(rc)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    _, _, chi0, _ = oracle_mod.moments(c.x, c.sigma)
    r = compare(out.cpu().numpy().T, ref, piv, chi0, tol=TOL)
    assert r["ok"], r
