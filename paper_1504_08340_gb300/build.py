"""Build the CUDA library libfwi.so in-tree for sm_103a (nvcc, no cmake)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libfwi.so")
SOURCES = ["fwi_api.cu", "fwi_kernels.cu", "fwi_stage.cu", "fwi_interior.cu", "fwi_pml.cu", "fwi_opt.cu", "fwi_noalloc.cu",
           "fwi_precond.cu", "fwi_conv_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


CHECK_LIB = os.path.join(HERE, "libfwi_check.so")  # the -DFWI_BOUNDS_CHECK build


def _stale(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), lib=LIB) -> str:
    if not force and not _stale(lib):
        return lib
    bdir = os.path.join(HERE, "_build" if lib == LIB else "_build_" + os.path.basename(lib).split(".")[0])
    os.makedirs(bdir, exist_ok=True)
    common = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", INCLUDE, "-I", CSRC, *extra]

    def compile_one(src):
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, lib)
    return lib


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checked library (every list-derived and tile-derived device index guarded,
    FWI_E_BOUNDS on a failed check), for tests; load it with FWI_LIBRARY=<path>."""
    return build(force, verbose, extra=("-DFWI_BOUNDS_CHECK",), lib=CHECK_LIB)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
    if "--checked" in sys.argv:
        print(build_checked(force="--force" in sys.argv, verbose=True))
