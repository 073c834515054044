"""The C ABI library loads, exports what the headers in include/ declare, and its host
logic (validation, grid sizing, kernel transform) is right -- no GPU needed."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import importlib
    importlib.import_module("paper_0901_1913_gb300.build").build()
    from paper_0901_1913_gb300 import _fc2
    return _fc2.load()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fc2_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_0901_1913_gb300 import _fc2
    for code in range(7):
        s = _fc2.status_string(code)
        assert s and s != "unknown status"


def test_grid_size(lib):
    assert lib.fc2_grid_size(16384, 2) == 32768
    assert lib.fc2_grid_size(1 << 22, 4) == 1 << 24
    assert lib.fc2_grid_size(1000, 2) == 2048
    assert lib.fc2_grid_size(10, 2) == 512        # minimum grid
    assert lib.fc2_grid_size(1 << 20, 1) == 0     # oversampling below 2
    assert lib.fc2_grid_size(1, 2) == 0


def test_kernel_transform_matches_quadrature(lib):
    """phihat(xi) = int phi(z) cos(2 pi xi z) dz of the spreading kernel, as
    used for deconvolution, against adaptive quadrature of the kernel itself."""
    from scipy.integrate import quad
    for w, os_ in [(7, 4), (9, 2), (12, 4), (14, 2)]:
        xi = np.array([0.0, 0.05, 0.1, 0.2, 0.25 if os_ == 2 else 0.125])
        got = np.zeros_like(xi)
        assert lib.fc2_kernel_ft(w, os_, xi.ctypes.data, xi.size, got.ctypes.data) == 0

        def phi(z):
            v = np.zeros(1)
            lib.fc2_kernel_eval(w, os_, np.array([z]).ctypes.data, 1, v.ctypes.data)
            return v[0]
        for k, x in enumerate(xi):
            ref, _ = quad(lambda z: phi(z) * math.cos(2 * math.pi * x * z), -w / 2, w / 2,
                          limit=200, epsabs=1e-14, epsrel=1e-13)
            assert got[k] == pytest.approx(ref, rel=1e-10), (w, os_, x)


def test_kernel_is_exponential_of_semicircle(lib):
    w, os_ = 8, 2
    beta = 0.97 * math.pi * (1 - 0.5 / os_) * w
    z = np.array([0.0, 1.0, 2.5, 3.99, 4.0, 5.0])
    out = np.zeros_like(z)
    lib.fc2_kernel_eval(w, os_, z.ctypes.data, z.size, out.ctypes.data)
    for zi, v in zip(z, out):
        s = 2 * zi / w
        ref = math.exp(beta * (math.sqrt(1 - s * s) - 1)) if abs(s) < 1 else 0.0
        assert v == pytest.approx(ref, rel=1e-14, abs=1e-300)


def test_default_widths(lib):
    assert lib.fc2_default_width(0, 2) > lib.fc2_default_width(1, 2)
    assert lib.fc2_default_width(0, 4) <= lib.fc2_default_width(0, 2)


@pytest.mark.parametrize("field,value", [("n", 0), ("H", 0), ("H", 17), ("df", 0.0),
                                         ("df", -1.0), ("f_min", -0.5), ("N", 1),
                                         ("oversample", 1), ("f_min", float("nan"))])
def test_validation_rejects_bad_arguments(lib, field, value):
    """Host-side validation runs before any device call."""
    from paper_0901_1913_gb300 import _fc2
    t = np.linspace(0, 10, 50)
    x = np.sin(t)
    s = np.full(50, 0.1)
    args = dict(n=50, H=3, f_min=0.1, df=0.01, N=100, oversample=2)
    args[field] = value
    opt = _fc2.make_options()
    h = ctypes.c_void_p()
    rc = lib.fc2_plan_create(t.ctypes.data, x.ctypes.data, s.ctypes.data, args["n"], args["H"],
                             args["f_min"], args["df"], args["N"], args["oversample"],
                             ctypes.byref(opt), ctypes.byref(h))
    assert rc == _fc2.FC2_ERR_INVALID_ARG
    assert not h.value


@pytest.mark.parametrize("kw", [dict(kernel_width=1), dict(kernel_width=17),
                                dict(kernel_width=40), dict(top_k=65), dict(oversample=1)])
def test_batched_validation_rejects_bad_options(lib, kw):
    """The batched entry point validates its options on the host before any
    device call (a spreading width beyond 16 cells would overrun the
    spreading kernels' key tables)."""
    from paper_0901_1913_gb300 import _fc2
    t = np.linspace(0, 10, 50)
    x = np.sin(t)
    s = np.full(50, 0.1)
    args = dict(oversample=2)
    args.update(kw)
    with pytest.raises(_fc2.Fc2Error) as ei:
        _fc2.execute_batched(np.array([0, 50]), t, x, s, np.array([3]), np.array([0.1]),
                             np.array([0.01]), np.array([100]), prec="mixed", **args)
    assert ei.value.code == _fc2.FC2_ERR_INVALID_ARG


def test_null_pointers_rejected(lib):
    from paper_0901_1913_gb300 import _fc2
    h = ctypes.c_void_p()
    rc = lib.fc2_plan_create(None, None, None, 10, 2, 0.1, 0.01, 100, 2, None, ctypes.byref(h))
    assert rc == _fc2.FC2_ERR_INVALID_ARG
    assert lib.fc2_execute(None, None, None, None, None) == _fc2.FC2_ERR_INVALID_ARG
    lib.fc2_plan_destroy(None)  # ignored


def test_product_path_does_not_use_the_oracle():
    """The package and the CUDA sources never import, link or read oracle/."""
    pkg = os.path.join(ROOT, "paper_0901_1913_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "fc2_oracle" not in txt and "fc2o_" not in txt, f


def test_batch_peak_records_layout_and_access():
    """The structured record type matches fc2_best byte for byte, and the
    batched peaks convert per curve, on access, to the single-curve dicts."""
    from paper_0901_1913_gb300 import _fc2
    assert _fc2.BEST_DTYPE.itemsize == ctypes.sizeof(_fc2.Best)
    for name, *_ in _fc2.Best._fields_:
        assert _fc2.BEST_DTYPE.fields[name][1] == getattr(_fc2.Best, name).offset, name
    rec = np.zeros((3, 2), dtype=_fc2.BEST_DTYPE)
    rec[1, 0]["j"], rec[1, 0]["f"], rec[1, 0]["dchi2"], rec[1, 0]["H"] = 7, 0.25, 3.5, 2
    rec[1, 0]["A"][:6] = [1, 2, 3, 4, 5, 6]
    # the same bytes read as the ctypes structure give the same dict
    ref = _fc2.Best.from_buffer_copy(rec[1, 0].tobytes()).as_dict()
    peaks = _fc2.BatchPeaks(rec)
    assert len(peaks) == 3 and [len(p) for p in peaks] == [2, 2, 2]
    got = peaks[1][0]
    assert {k: got[k] for k in ("j", "f", "dchi2", "H", "flags")} == \
        {k: ref[k] for k in ("j", "f", "dchi2", "H", "flags")}
    np.testing.assert_array_equal(got["A"], ref["A"])
    assert got["A"].tolist() == [1, 2, 3, 4, 5]  # 2H + 1 coefficients
    assert [p[0]["j"] for p in peaks[0:3:2]] == [0, 0]
