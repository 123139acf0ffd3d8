"""Build the sm_103a CUDA library libhr2.so in-tree (nvcc, no JIT cache).

Usage: python -m paper_1910_01070_b300.build [--force] [--bounds-check]
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhr2.so")
# the bounds-checked build (index checks that report HR2_EBOUNDS instead of
# touching memory outside a buffer): a debugging aid, built beside the library
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libhr2_bounds.so")
# (source, object, extra defines): the FP32 forward kernel's instantiations are
# compiled once per angle-node count, first, since they take longest
UNITS = [("kern_fwd32_inst.cu", "kern_fwd32_n%d.o" % n, ["-DHR2_FWD32_NMU=%d" % n]) for n in range(1, 9)] + [
    (src, src.replace(".cu", ".o"), [])
    for src in ("kern_forward.cu", "kern_nested.cu", "kern_setup.cu", "kern_peaks.cu", "api.cu")]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "hr2.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _unit_deps(src: str) -> float:
    """Newest of a unit's source, every header and this script (a header change rebuilds all)."""
    files = [os.path.join(CSRC, src), os.path.join(INCLUDE, "hr2.h"), __file__]
    files += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, bounds_check: bool = False) -> str:
    lib_path, build_dir = (LIB_BOUNDS, BUILD_BOUNDS) if bounds_check else (LIB, BUILD)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= _deps():
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    if bounds_check:
        extra.append("-DHR2_BOUNDS_CHECK=1")

    def compile_one(unit):
        src, obj, defines = unit
        obj = os.path.join(build_dir, obj)
        if not force and os.path.exists(obj) and os.path.getmtime(obj) >= _unit_deps(src):
            return obj
        cmd = [NVCC, *ARCH, *FLAGS, *defines, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose or ptxas_info:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(UNITS), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib_path + ".tmp.%d" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                bounds_check="--bounds-check" in sys.argv))
