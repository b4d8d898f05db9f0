"""Build libpflbm.so (the CUDA library behind include/pflbm.h) in-tree.

Compiles each ``csrc/*.cu`` for sm_103a in parallel and links a shared
library next to this file, and beside it libpflbm_bounds.so, the
index-checked debug build (the step kernels and the entry points compiled
with -DPFLBM_BOUNDS, everything else shared).
``python -m paper_2312_00369_gb300.build``.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpflbm.so")
LIB_BOUNDS = os.path.join(HERE, "libpflbm_bounds.so")
# translation units whose accesses the index-checked build checks
BOUNDS_SRCS = ("step.cu", "step2.cu", "step_tma.cu", "capi.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit multiply-add contraction; the kernels write their
# fused multiply-adds explicitly, so every kernel that inlines a formula
# rounds it the same way
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-fmad=false",
         "-Xptxas", "-v"] + ARCH


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return path


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(HERE, "..", "include", "*.h")))


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(LIB_BOUNDS):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_BOUNDS))
    return any(os.path.getmtime(f) > t for f in _sources() + _headers() + [__file__])


def _compile(job):
    src, bounds = job
    obj = os.path.join(OBJ, os.path.basename(src) + (".bounds.o" if bounds else ".o"))
    cmd = [nvcc()] + FLAGS + (["-DPFLBM_BOUNDS"] if bounds else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = _sources()
    jobs = [(s, False) for s in srcs] + [(s, True) for s in srcs if os.path.basename(s) in BOUNDS_SRCS]
    # the largest translation units first
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        results = dict(zip(jobs, ex.map(_compile, jobs)))
    if verbose:
        for _, log in results.values():
            sys.stderr.write(log)
    for out, bounds in ((LIB, False), (LIB_BOUNDS, True)):
        objs = [results[(s, bounds and os.path.basename(s) in BOUNDS_SRCS)][0] for s in srcs]
        tmp = out + ".tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
