"""fc2_dchi2_exact_noalloc: the allocation-free exact evaluation.

For callers that cannot allocate device memory when they need an answer (their
memory is reserved by another allocator, or an allocation's implicit
synchronisation is not acceptable), this entry point keeps its intermediates
in a fixed-size device array owned by the library.  It must give the same
Delta chi^2 as the regular entry point, call after call.
"""
import ctypes

import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import TOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_execute_twice():
    import torch

    from paper_0901_1913_gb300 import _fc2
    lib = _fc2.load()
    lib.fc2_dchi2_exact_noalloc.argtypes = [ctypes.c_void_p] * 3 + [
        ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
        ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    lib.fc2_dchi2_exact_noalloc.restype = ctypes.c_int

    c = synth.short_curve()
    d_ref, best, _, chi0 = _fc2.periodogram(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "fp64")
    rng = np.random.default_rng(4)
    bins = np.unique(np.concatenate([[b["j"] for b in best],
                                     rng.choice(c.N, 120, replace=False)]))[:128]
    dev = torch.device("cuda", 0)
    t = torch.from_numpy(c.t).to(dev)
    x = torch.from_numpy(c.x).to(dev)
    s = torch.from_numpy(c.sigma).to(dev)
    b = torch.from_numpy(bins.astype(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    outs = []
    for _ in range(2):
        out = torch.full((c.H, bins.size), float("nan"), dtype=torch.float64, device=dev)
        rc = lib.fc2_dchi2_exact_noalloc(t.data_ptr(), x.data_ptr(), s.data_ptr(), c.n, c.H,
                                         c.f_min, c.df, b.data_ptr(), bins.size, out.data_ptr(),
                                         stream)
        assert rc == 0, _fc2.status_string(rc)
        outs.append(out.cpu().numpy())
    for o in outs:
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - d_ref[:, bins])) <= TOL * chi0
    np.testing.assert_array_equal(outs[0], outs[1])
    # sizes beyond the fixed scratch are refused
    rc = lib.fc2_dchi2_exact_noalloc(t.data_ptr(), x.data_ptr(), s.data_ptr(), c.n, c.H, c.f_min,
                                     c.df, b.data_ptr(), 129, out.data_ptr(), stream)
    assert rc == _fc2.FC2_ERR_INVALID_ARG
