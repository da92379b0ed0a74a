"""In-tree build of the CUDA library ``libgpe.so`` for sm_103a.

Each ``csrc/*.cu`` translation unit is compiled in parallel with nvcc, then
linked into one shared library next to this file.  No cmake, no torch
extension machinery: the library has a plain C ABI (``include/gpe.h``).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libgpe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fno-gnu-unique: statics of inline functions and templates stay this library's
# own, so that two copies of it (libgpe.so, libgpe_check.so) in one process
# never share one
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xcompiler", "-fno-gnu-unique",
         "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(HERE, "csrc")]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgpe.so")


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


# the checking build: index checks in the kernels, guard bands around buffers
CHECK_LIB = os.path.join(HERE, "libgpe_check.so")
VARIANTS = ((LIB, "_build", []), (CHECK_LIB, "_build_check", ["-DGPE_BOUNDS_CHECK"]))


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(HERE, "csrc", "*.cuh")) + glob.glob(os.path.join(HERE, "csrc", "*.h")) + \
        glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Builds libgpe.so and libgpe_check.so (every translation unit of both in
    one parallel pool); returns the path of libgpe.so."""
    todo = [v for v in VARIANTS if force or _stale(v[0])]
    if not todo:
        return LIB
    nvcc = _nvcc()
    srcs = sources()
    jobs = []
    for lib, objname, extra in todo:
        objdir = os.path.join(HERE, objname)
        os.makedirs(objdir, exist_ok=True)
        for src in srcs:
            jobs.append((src, os.path.join(objdir, os.path.basename(src)[:-3] + ".o"), extra))

    def compile_one(job):
        src, obj, extra = job
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {' '.join(extra)}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    # the slowest translation units first, so that they do not end the build alone
    jobs.sort(key=lambda j: -os.path.getsize(j[0]) - (10 ** 6 if "gpe_step" in j[0] else 0))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, jobs))
    for lib, objname, extra in todo:
        mine = [o for o in objs if os.sep + objname + os.sep in o]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + mine + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
