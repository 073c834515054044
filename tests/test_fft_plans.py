"""Transform pass plans against what the pass kernels assume, on the host.

The kernels store a non-last pass's tile as rows of the next pass's tiles, Jn
columns at a time; with Jn above the current radix R a tile's store walks past
its R rows, out of its shared memory and out of the grid.  Such plans (a small
radix followed by a larger one, as unbalanced three-pass splits produce) are
refused by the library; every plan it uses -- the fixed planner's and the
autotuner's candidates, for every grid length, both precisions and every float
kernel family -- replays in range with the kernels' own index functions.
"""
import ctypes
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import importlib
    importlib.import_module("paper_0901_1913_gb300.build").build()
    from paper_0901_1913_gb300 import _fc2
    L = _fc2.load()
    L.fc2_debug_fft_plan.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.fc2_debug_fft_plan.restype = ctypes.c_int
    L.fc2_debug_fft_candidates.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int]
    L.fc2_debug_fft_candidates.restype = ctypes.c_int
    L.fc2_debug_fft_plan_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p]
    L.fc2_debug_fft_plan_check.restype = ctypes.c_int
    return L


def check(lib, logM, fp64, kern, rs, validate=True):
    r = np.ascontiguousarray(rs, dtype=np.int32)
    info = np.zeros(4, dtype=np.int64)
    rc = lib.fc2_debug_fft_plan_check(logM, fp64, kern, r.ctypes.data, r.size, int(validate),
                                      info.ctypes.data)
    return rc, info


def library_plans(lib, logM, fp64):
    out = np.zeros(8, dtype=np.int32)
    P = lib.fc2_debug_fft_plan(logM, fp64, out.ctypes.data, 8)
    plans = [list(out[:P])]
    buf = np.zeros(64, dtype=np.int32)
    n = lib.fc2_debug_fft_candidates(logM, fp64, buf.ctypes.data, 64)
    assert n > 0
    i = 0
    while i < n:
        P = int(buf[i])
        plans.append(list(buf[i + 1:i + 1 + P]))
        i += 1 + P
    return plans


@pytest.mark.parametrize("fp64", [0, 1])
def test_every_library_plan_replays_in_range(lib, fp64):
    for logM in range(9, 29):
        for rs in library_plans(lib, logM, fp64):
            assert sum(rs) == logM
            for kern in (1, 2, 3, 4, 5):
                rc, info = check(lib, logM, fp64, kern, rs)
                assert rc == 0, (logM, fp64, kern, rs, rc, info)


def test_small_radix_before_larger_is_refused_and_would_store_out_of_range(lib):
    # the shape of the recorded autotuner fault: a 2^20-point plan split
    # unevenly into three passes with radices down to 2^5
    rc, _ = check(lib, 20, 0, 1, [5, 7, 8])
    assert rc == 1
    rc, info = check(lib, 20, 0, 1, [5, 7, 8], validate=False)
    assert rc != 0 and info[0] == 0          # the first pass's store toward the second
    assert info[1] in (7, 8)                 # tile row past R, or a global index past M


@pytest.mark.parametrize("fp64", [0, 1])
def test_validity_implies_in_range_for_all_splits(lib, fp64):
    """Every two- and three-pass split with radices 2^5..2^12 and every kernel
    family: a plan the validator accepts replays in range, and every plan it
    refuses for the tile-width rule does go out of range."""
    seen_bad = 0
    for logM in range(13, 29, 3):
        for P in (2, 3):
            for rs in itertools.product(range(5, 13), repeat=P):
                if sum(rs) != logM:
                    continue
                for kern in (1, 2, 3, 4, 5):
                    rc_v, _ = check(lib, logM, fp64, kern, rs)
                    rc_r, info = check(lib, logM, fp64, kern, rs, validate=False)
                    if rc_v == 0:
                        assert rc_r == 0, (logM, rs, kern, info)
                    elif rc_r != 0:
                        seen_bad += 1
    assert seen_bad > 0
