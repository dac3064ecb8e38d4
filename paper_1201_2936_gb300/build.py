"""Build libqh.so (the CUDA library behind include/qh.h) in-tree with nvcc.

Every translation unit is compiled for sm_103a only, in parallel, and linked
into paper_1201_2936_gb300/_build/libqh.so.  The CUDA runtime is linked
statically so the library shares only the driver context with PyTorch.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
# QH_DEBUG_BUILD=1 selects the checked build (-DQH_DEBUG=1: device-side
# alignment and bounds checks, read with qh_debug_checks) in its own folder
DEBUG = os.environ.get("QH_DEBUG_BUILD", "") == "1"
BUILD = os.path.join(HERE, "_build_debug" if DEBUG else "_build")
LIB = os.path.join(BUILD, "libqh.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqh")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(objs) -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps += glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    if not force and not _stale(objs):
        return LIB
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if DEBUG:
        flags += ["-DQH_DEBUG=1"]
    # tuning knobs (e.g. -DQH2D_SITEMS=4 -DQH2D_MINBLOCKS=3); a change needs force=True
    flags += os.environ.get("QH_NVCC_EXTRA", "").split()
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc()] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
