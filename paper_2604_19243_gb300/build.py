"""In-tree build of libfmm.so for sm_103a (nvcc for the CUDA sources, g++ for the host C++), and of
its bounds-checked twin libfmm_debug.so (the same sources with FMM_DEBUG defined).

`python -m paper_2604_19243_gb300.build` or `build()`; objects and the library go to
paper_2604_19243_gb300/_build/.  Translation units compile in parallel; a unit is rebuilt
when it or any header of csrc/ is newer than its object.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfmm.so")
LIB_DEBUG = os.path.join(OUT, "libfmm_debug.so")   # FMM_DEBUG: in-kernel bounds checks
ROOT = os.path.dirname(HERE)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Per-file flags.  The near-field kernel flushes denormals: squared distances between distinct
# FP32 points are never denormal (coincident pairs are skipped explicitly), so rsqrtf needs no
# range fix-up around the hardware reciprocal square root.
EXTRA = {"p2p.cu": ["-ftz=true"]}


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found")


def _stale(obj, src, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + headers + [os.path.abspath(__file__)])


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stderr


def _build_lib(nvcc, cuda, out, lib, defines, headers, verbose, force):
    os.makedirs(out, exist_ok=True)
    jobs, objs = [], []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        obj = os.path.join(out, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, src, headers):
            jobs.append([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *defines,
                         *EXTRA.get(os.path.basename(src), []),
                         "-Xptxas", "-v" if verbose else "-O3", "-c", src, "-o", obj])
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cpp"))):
        obj = os.path.join(out, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, src, headers):
            jobs.append(["g++", "-O2", "-fPIC", "-std=c++17", "-pthread", *defines,
                         "-I" + os.path.join(cuda, "include"), "-c", src, "-o", obj])
    return jobs, objs, lib


def build(verbose: bool = False, force: bool = False) -> str:
    """Builds libfmm.so and the bounds-checked libfmm_debug.so (FMM_DEBUG); returns the former."""
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    libs = [_build_lib(nvcc, cuda, OUT, LIB, [], headers, verbose, force),
            _build_lib(nvcc, cuda, os.path.join(OUT, "debug"), LIB_DEBUG, ["-DFMM_DEBUG"], headers, verbose, force)]
    jobs = [j for js, _, _ in libs for j in js]
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for log in ex.map(_compile, jobs):
                if verbose and log:
                    print(log)
    for js, objs, lib in libs:
        if js or not os.path.exists(lib):
            tmp = lib + f".tmp{os.getpid()}"
            _compile([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
