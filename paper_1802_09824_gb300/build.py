"""Compile libphpp.so (the CUDA library behind include/phpp.h) for sm_103a.

Each .cu file under csrc/ is compiled in parallel with nvcc into _build/,
then linked into paper_1802_09824_gb300/libphpp.so.  Objects are rebuilt
only when a source or header is newer than the object.  `--checked` (or
build(checked=True)) makes libphpp_checked.so from the same sources with the
debug bounds checks of csrc/checks.cuh compiled in (objects in
_build/checked/).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libphpp.so")
CHECKED_OUT = os.path.join(HERE, "libphpp_checked.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code is compiled without floating-point contraction, so host-side
# decisions (domain cells, tables) round the same on x86 and Arm
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _newest_header() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src: str, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(BUILD, "checked" if checked else "", os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), _newest_header()):
        return obj
    cmd = [_nvcc(), *ARCH, *NVCC_FLAGS, *(["-DPHPP_BOUNDS_CHECK"] if checked else []), "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(verbose: bool = False, checked: bool = False) -> str:
    os.makedirs(os.path.join(BUILD, "checked") if checked else BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, checked), srcs))
    out = CHECKED_OUT if checked else OUT
    if (not os.path.exists(out)) or os.path.getmtime(out) < max(os.path.getmtime(o) for o in objs):
        libdir = os.path.join(os.path.dirname(os.path.dirname(_nvcc())), "lib64")
        cmd = [_nvcc(), *ARCH, "-shared", *objs, "-o", out + ".tmp", "-lcudart", "-lcufft",
               "-Xlinker", "-rpath", "-Xlinker", libdir]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, checked="--checked" in sys.argv))
