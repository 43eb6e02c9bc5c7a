"""Build the CUDA library (sm_103a) in-tree: paper_2206_15454_b300/_lib/liblbm_b300.so.

nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo.  Division and square
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
    return sources() + sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh"))) + [
        os.path.join(ROOT, "include", "lbm.h"), os.path.abspath(__file__)]


# The checked build: every bulk copy and global store of the step is verified
# against its buffer (LBM_CHECK_BOUNDS); used by the tests, never by default.
LIB_CHECKED = os.path.join(OUT_DIR, "liblbm_b300_checked.so")


def _command(out: str, checked: bool, verbose: bool) -> list:
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
           "-prec-div=false", "-prec-sqrt=false",
           "-Xcompiler", "-fPIC", "-shared", "-cudart", "static",
           "-I", os.path.join(ROOT, "include"), "-o", out, *sources()]
    if checked:
        cmd.insert(1, "-DLBM_CHECK_BOUNDS")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def _fresh(path: str) -> bool:
    return os.path.exists(path) and os.path.getmtime(path) >= max(os.path.getmtime(p) for p in deps())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build the library (or, with checked=True, the checked build) in-tree."""
    out = LIB_CHECKED if checked else LIB
    if not force and _fresh(out):
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    subprocess.run(_command(out, checked, verbose), check=True)
    return out


def build_all(force: bool = False) -> None:
    """Both builds, compiled side by side."""
    os.makedirs(OUT_DIR, exist_ok=True)
    procs = [subprocess.Popen(_command(out, checked, False))
             for out, checked in ((LIB, False), (LIB_CHECKED, True))
             if force or not _fresh(out)]
    for p in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, p.args)


if __name__ == "__main__":
    if "--all" in sys.argv:
        build_all(force="--force" in sys.argv)
    else:
        print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                    checked="--checked" in sys.argv))
