"""Build libgwx.so in-tree for sm_103a with nvcc (no CMake, no torch extension machinery).

Each CUDA translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and the objects are
linked into ``paper_2407_19048_gb300/libgwx.so``.  A rebuild is skipped when the
library is newer than every source file.

Usage: ``python -m paper_2407_19048_gb300.build [--force] [--verbose] [--debug]``
(``--debug``: ``libgwx_debug.so`` with index checks, loaded when GWX_DEBUG=1).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgwx.so")
# the debug build: the same sources with GWX_DEBUG_CHECKS (index checks on the hot
# kernels' global accesses, recorded for gwx_debug_status instead of faulting)
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libgwx_debug.so")
UNITS = ["capi.cu", "k_random.cu", "k_spectral.cu", "k_waveform.cu", "k_fused.cu", "k_weights.cu", "k_gemm.cu", "k_dense.cu", "k_learn.cu", "k_noalloc.cu", "k_flow.cu", "k_flow_fused.cu", "k_skymap.cu", "k_vicreg.cu", "k_resnet.cu", "k_conv.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: libgwx needs the CUDA toolkit to build")
    return exe


def sources():
    out = [os.path.join(CSRC, u) for u in UNITS]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out.append(os.path.join(INCLUDE, "gwx.h"))
    return out


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force=False, verbose=False, extra_flags=(), debug=False):
    """Compile and link libgwx.so (debug: libgwx_debug.so with GWX_DEBUG_CHECKS); returns
    its path."""
    lib_path, build_dir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if debug:
        extra_flags = ("-DGWX_DEBUG_CHECKS", *extra_flags)
    if not force and up_to_date(lib_path):
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    exe = nvcc()

    def compile_one(unit):
        obj = os.path.join(build_dir, unit.replace(".cu", ".o"))
        cmd = [exe, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, unit), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = lib_path + ".tmp"
    cmd = [exe, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv, debug="--debug" in sys.argv))
