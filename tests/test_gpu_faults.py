"""Failure detection without a GPU fault.

* Allocation failures are injected on the host: the library's pool is told to
  fail its k-th allocation (fc2_debug_fail_alloc) for every allocation a plan
  creation or a batched call makes.  Each attempt must end in FC2_ERR_OOM (or
  succeed, when the failed allocation was a best-effort cache), leave no
  device memory behind, and the next normal call must give the same results.
* A bounded device-side wait is made to run out: the bulk-copy transform pass
  arms the mbarrier of one tile but never issues its copy (fc2_debug_fault),
  with a wait limit of about a millisecond.  The CTA gives up, waits (bounded)
  for its other copies and returns; fc2_execute returns FC2_ERR_TIMEOUT and the
  plan's next execute is correct.  No kernel traps, faults or spins unbounded.
"""
import numpy as np
import pytest

from paper_0901_1913_gb300 import synth
from tests.parity import TOL, compare

pytestmark = pytest.mark.gpu


def test_plan_creation_survives_each_failed_allocation():
    from paper_0901_1913_gb300 import _fc2
    lib = _fc2.load()
    c = synth.short_curve(n=400, N=2048)
    args = (c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, 2, "mixed")
    d_ref, _, _, _ = _fc2.periodogram(*args)   # warms the pool and the table cache
    base = lib.fc2_debug_pool_used(0)
    a0 = lib.fc2_debug_alloc_count()
    _fc2.Plan(*args).close()
    nalloc = lib.fc2_debug_alloc_count() - a0
    assert nalloc >= 10
    oom = 0
    try:
        for k in range(1, nalloc + 1):
            lib.fc2_debug_fail_alloc(k)
            try:
                p = _fc2.Plan(*args)
            except _fc2.Fc2Error as e:
                assert e.code == _fc2.FC2_ERR_OOM, (k, e)
                oom += 1
            else:  # a best-effort allocation failed: the plan still works
                with p:
                    d, _, _, _ = p.execute()
                np.testing.assert_array_equal(d, d_ref)
            lib.fc2_debug_fail_alloc(0)
            assert lib.fc2_debug_pool_used(0) == base, k
    finally:
        lib.fc2_debug_fail_alloc(0)
    assert oom >= nalloc - 2
    d, _, _, _ = _fc2.periodogram(*args)
    np.testing.assert_array_equal(d, d_ref)


def test_batched_call_survives_each_failed_allocation():
    from paper_0901_1913_gb300 import _fc2
    lib = _fc2.load()
    b = synth.survey_batch(C=6, N=1 << 12)
    args = (b.offsets, b.t, b.x, b.sigma, b.H, b.f_min, b.df, b.N, b.oversample, "mixed")
    ref, pk_ref, _ = _fc2.execute_batched(*args)
    base = lib.fc2_debug_pool_used(0)
    a0 = lib.fc2_debug_alloc_count()
    _fc2.execute_batched(*args)
    nalloc = lib.fc2_debug_alloc_count() - a0
    assert nalloc >= 10
    oom = 0
    try:
        for k in range(1, nalloc + 1):
            lib.fc2_debug_fail_alloc(k)
            try:
                got, _, _ = _fc2.execute_batched(*args)
            except _fc2.Fc2Error as e:
                assert e.code == _fc2.FC2_ERR_OOM, (k, e)
                oom += 1
            else:
                np.testing.assert_array_equal(got, ref)
            lib.fc2_debug_fail_alloc(0)
            assert lib.fc2_debug_pool_used(0) == base, k
    finally:
        lib.fc2_debug_fail_alloc(0)
    assert oom >= nalloc - 2
    got, pk, _ = _fc2.execute_batched(*args)
    np.testing.assert_array_equal(got, ref)
    np.testing.assert_array_equal(pk.records, pk_ref.records)


def test_bounded_wait_gives_up_and_reports_timeout(oracle_mod):
    from paper_0901_1913_gb300 import _fc2
    # M = 2^18 (N = 2^16, 4x oversampled): two passes of radix 2^9 with the
    # bulk-copy kernel family; the second pass streams its tiles into shared
    # memory with bulk copies on mbarriers
    c = synth.long_curve(n=3000, N=1 << 16)
    with _fc2.Plan(c.t, c.x, c.sigma, c.H, c.f_min, c.df, c.N, c.oversample, "mixed",
                   fft_kernel="bulk") as p:
        d0, _, _, chi0 = p.execute()
        p.debug_fault(wait_cycles=2_000_000, drop_tile=0)   # ~1 ms per wait
        with pytest.raises(_fc2.Fc2Error) as ei:
            p.execute()
        assert ei.value.code == _fc2.FC2_ERR_TIMEOUT
        p.debug_fault(0, -1)
        d1, _, _, _ = p.execute()
    np.testing.assert_array_equal(d1, d0)
    bins = np.arange(0, c.N, 257)
    ref, piv = oracle_mod.dchi2_bins(c.t, c.x, c.sigma, c.H, c.f_min, c.df, bins,
                                     with_pivots=True)
    r = compare(d1[:, bins].T, ref, piv, chi0, tol=TOL)
    assert r["ok"], r
