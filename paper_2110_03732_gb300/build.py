"""Build of the CUDA library ``libgrmhd.so`` (sm_103a) with nvcc, in-tree.

Each ``csrc/*.cu`` compiles to an object in parallel, then one shared library is
linked into ``_build/``.  No cmake and no torch extension machinery: the library is
a plain C ABI (``include/grmhd.h``).

``build(checked=True)`` also builds the bounds-checked copy of the library
(``_build_checked/libgrmhd.so``, compiled with ``-DGRMHD_CHECK_BOUNDS``): every array
index its kernels form is checked and counted when it leaves the array
(``grmhd_bounds_violations``).  Both copies compile in one job pool.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgrmhd.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libgrmhd.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force: bool = False, ptxas_verbose: bool = False, checked: bool = False) -> str:
    """Compile every kernel source for sm_103a and link ``_build/libgrmhd.so`` (and,
    with ``checked``, the bounds-checked copy).  Returns the normal library's path."""
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "grmhd.h")]
    nvcc = _nvcc()
    variants = [(BUILD, LIB, [])]
    if checked:
        variants.append((BUILD_CHECKED, LIB_CHECKED, ["-DGRMHD_CHECK_BOUNDS"]))
    jobs, links = [], []
    for bdir, lib, extra in variants:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
                if ptxas_verbose:
                    cmd.insert(1, "-Xptxas=-v")
                jobs.append(cmd)
        links.append((lib, objs))
    logs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, len(jobs)))) as ex:
        for out in ex.map(_run, jobs):
            logs.append(out)
    for lib, objs in links:
        if jobs or force or _stale(lib, objs):
            tmp = lib + f".{os.getpid()}.tmp"
            _run([nvcc, *ARCH, "-shared", *objs, "-o", tmp, "-lcudart"])
            os.replace(tmp, lib)
    if ptxas_verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv, checked="--checked" in sys.argv))
