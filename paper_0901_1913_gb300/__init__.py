"""GB300 (sm_103a) Fast chi-squared periodogram (Palmer 2009, arXiv 0901.1913).

The compute path is libfc2.so (hand-written CUDA behind a C ABI, include/fc2.h);
this package holds its ctypes binding, the in-tree build and the seeded
synthetic workloads.  Importing it does not load the library; the first call
that needs it does, and raises if it has not been built.
"""
from . import synth  # noqa: F401


def build(verbose: bool = False) -> str:
    from .build import build as _b
    return _b(verbose)


def __getattr__(name):
    if name in ("Plan", "periodogram", "load", "Fc2Error", "make_options", "Best", "Options"):
        from . import _fc2
        return getattr(_fc2, name)
    raise AttributeError(name)
