"""Build the in-tree C-ABI library ``libgbri.so`` for sm_103a with nvcc (no cmake).

Every ``csrc/*.cu`` file is compiled in parallel to an object under ``_build/``
and linked with cuFFT into ``paper_1903_04502_gb300/libgbri.so``.  ``debug=True``
builds the same sources with ``-DGBRI_DEBUG`` (bounds checks in the visibility
kernels that record into a per-plan error word) into ``_build_debug/`` and
``libgbri_debug.so``, which the binding loads when ``GBRI_DEBUG_LIB=1``.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libgbri.so")
BUILD_DEBUG = os.path.join(ROOT, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libgbri_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand) and shutil.which(cand) is None:
        raise RuntimeError("nvcc not found")
    return cand


def cuda_home():
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))


FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
         "--expt-relaxed-constexpr", "-I" + os.path.join(ROOT, "include")]


def _compile(src, build_dir=BUILD, extra=()):
    obj = os.path.join(build_dir, os.path.basename(src) + ".o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(
            os.path.getmtime(f) for f in _deps(src)):
        return obj
    cmd = [nvcc()] + ARCH + FLAGS + list(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stdout + r.stderr))
    return obj


def _deps(src):
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hdrs.append(os.path.join(ROOT, "include", "gbri.h"))
    return [src] + hdrs


def build(verbose=False, debug=False):
    build_dir, lib_out = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    extra = ("-DGBRI_DEBUG",) if debug else ()
    os.makedirs(build_dir, exist_ok=True)
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    with cf.ThreadPoolExecutor(max_workers=min(16, len(srcs))) as ex:
        objs = list(ex.map(lambda f: _compile(f, build_dir, extra), srcs))
    lib_dir = os.path.join(cuda_home(), "lib64")
    if not os.path.isdir(lib_dir):
        lib_dir = os.path.join(cuda_home(), "lib")
    newest = max(os.path.getmtime(o) for o in objs)
    if os.path.exists(lib_out) and os.path.getmtime(lib_out) >= newest:
        return lib_out
    cmd = [nvcc()] + ARCH + ["-shared", "-o", lib_out + ".tmp"] + objs + [
        "-L" + lib_dir, "-lcufft", "-Xlinker", "-rpath," + lib_dir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stdout + r.stderr))
    os.replace(lib_out + ".tmp", lib_out)
    if verbose:
        print("built", lib_out)
    return lib_out


def build_all(verbose=False):
    """The default library and the bounds-checked one, compiled side by side."""
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        futs = [ex.submit(build, verbose, False), ex.submit(build, verbose, True)]
        return [f.result() for f in futs]


if __name__ == "__main__":
    build_all(verbose=True)
    sys.exit(0)
