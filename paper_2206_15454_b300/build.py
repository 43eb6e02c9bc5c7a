"""Build the CUDA library (sm_103a) in-tree: paper_2206_15454_b300/_lib/liblbm_b300.so.

nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo, one object per
translation unit of csrc/ (compiled in parallel under _build/), linked into
one shared library.  Division and square
root use the approximate hardware forms (-prec-div=false -prec-sqrt=false,
about 2 ulp); denormals and all other FP32 rounding stay IEEE (no -use_fast_math),
which keeps the FP32 path within 1e-6 of the FP64 oracle.  The runtime is
linked statically.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblbm_b300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + sorted(
        glob.glob(os.path.join(HERE, "csrc", "*.h"))) + sorted(
        glob.glob(os.path.join(HERE, "csrc", "*.inc"))) + [
        os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]


# The checked build: every bulk copy and global store of the step is verified
# against its buffer (LBM_CHECK_BOUNDS); used by the tests, never by default.
LIB_CHECKED = os.path.join(OUT_DIR, "liblbm_b300_checked.so")
OBJ_DIR = os.path.join(ROOT, "_build")

FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-prec-div=false",
         "-prec-sqrt=false", "-Xcompiler", "-fPIC"]


def _jobs(out: str, checked: bool, verbose: bool):
    """(compile commands, link command): every translation unit of csrc/ to an
    object of its own (compiled in parallel), then one shared library."""
    tag = "checked" if checked else "plain"
    objs, compiles = [], []
    for src in sources():
        obj = os.path.join(OBJ_DIR, tag, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if checked:
            cmd.insert(1, "-DLBM_CHECK_BOUNDS")
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        compiles.append(cmd)
    link = [NVCC, *ARCH, "-shared", "-cudart", "static", "-o", out, *objs]
    return compiles, link


def _fresh(path: str) -> bool:
    return os.path.exists(path) and os.path.getmtime(path) >= max(os.path.getmtime(p) for p in deps())


def _run_all(cmds):
    procs = [subprocess.Popen(c) for c in cmds]
    bad = [p for p in procs if p.wait() != 0]
    if bad:
        raise subprocess.CalledProcessError(bad[0].returncode, bad[0].args)


def _build(targets, verbose=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = [_jobs(out, checked, verbose) for out, checked in targets]
    for compiles, _ in jobs:
        for c in compiles:
            os.makedirs(os.path.dirname(c[c.index("-o") + 1]), exist_ok=True)
    _run_all([c for compiles, _ in jobs for c in compiles])
    _run_all([link for _, link in jobs])


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the library (or, with checked=True, the checked build) in-tree."""
    out = LIB_CHECKED if checked else LIB
    if not force and _fresh(out):
        return out
    _build([(out, checked)], verbose)
    return out


def build_all(force: bool = False) -> None:
    """Both builds, their translation units compiled side by side."""
    targets = [(out, checked) for out, checked in ((LIB, False), (LIB_CHECKED, True))
               if force or not _fresh(out)]
    if targets:
        _build(targets)


if __name__ == "__main__":
    if "--all" in sys.argv:
        build_all(force="--force" in sys.argv)
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                    checked="--checked" in sys.argv))
