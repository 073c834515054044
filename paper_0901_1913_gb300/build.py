"""Build libfc2.so (sm_103a) in-tree with nvcc: one object per source, compiled
in parallel, then linked as a shared library next to this file."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfc2.so")
SOURCES = ["fc2_api.cu", "k_prep.cu", "k_fft.cu", "k_solve.cu", "k_batch.cu", "k_adjoint.cu",
           "k_signif.cu", "k_trend.cu", "fc2_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


# Sources that embed the version of all sources (the batched path's tuning
# cache file keys its entries by it): rebuilt whenever any source changes.
VERSIONED = ("k_batch.cu",)


def _compile(src: str, verbose: bool) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(BUILD, src + ".o")
    deps = [path] + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    inc = os.path.join(HERE, "..", "include")
    deps += [os.path.join(inc, h) for h in os.listdir(inc) if h.endswith(".h")]
    defs = []
    stamp = None
    if src in VERSIONED:
        ver = sources_version()
        defs = [f'-DFC2_SRC_VERSION="{ver}"']
        stamp = obj + ".ver"
    fresh = os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(d) for d in deps)
    if fresh and stamp is not None:
        try:
            with open(stamp) as fh:
                fresh = fh.read().strip() == ver
        except OSError:
            fresh = False
    if fresh:
        return obj
    cmd = [nvcc(), "-c", path, "-o", obj, "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
           "-lineinfo", "--expt-relaxed-constexpr"] + defs + ARCH
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    if stamp is not None:
        with open(stamp, "w") as fh:
            fh.write(ver)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with ThreadPoolExecutor(len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB



def sources_version() -> str:
    """Short hash of every library source and public header; whole-pipeline
    profiles record it so that stale counters are recognised after any kernel
    changes."""
    import hashlib
    h = hashlib.sha1()
    inc = os.path.join(HERE, "..", "include")
    files = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                   if f.endswith((".cu", ".cuh", ".h", ".cpp")))
    files += sorted(os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h"))
    for f in files:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def kernel_version() -> str:
    """Short hash of the transform sources; profiles record it so that stale
    counters are recognised after the kernel changes."""
    import hashlib
    h = hashlib.sha1()
    for f in ("k_fft.cu", "fc2_common.cuh"):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
