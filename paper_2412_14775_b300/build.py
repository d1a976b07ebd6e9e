"""Compile the sm_103a CUDA library in-tree: paper_2412_14775_b300/_lib/librfi.so.

nvcc cross-compiles for sm_103a without a GPU.  The CUDA runtime is linked
statically, so the library loads (and exports its C ABI) on a host without a GPU
driver; CUDA is only initialised by the first call that needs a device.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "_lib", "librfi.so")
SOURCES = ["rfi_api.cu", "rfi_inst_f32.cu", "rfi_inst_f16.cu", "rfi_inst_pw_f32.cu",
           "rfi_inst_pw_f16.cu", "rfi_inst_ad_f32.cu", "rfi_inst_ad_f16.cu", "rfi_inst_pf_f32.cu",
           "rfi_inst_pf_f16.cu", "rfi_inst_tma_f32.cu", "rfi_inst_tma_f16.cu", "rfi_adapt.cu",
           "rfi_noalloc.cu", "rfi_inst_sw_f32.cu", "rfi_inst_sw_f16.cu",
           "rfi_inst_wp_f32.cu", "rfi_inst_wp_f16.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--cudart", "static", "-I", INCLUDE, "-I", CSRC]


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "rfi.h"))
    return files


# The debug-bounds build: every global access of the kernels checked against its
# buffer's extent (violations are skipped and reported by rfi_check).
DEBUG_LIB = os.path.join(HERE, "_lib", "librfi_debug.so")


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    """Compile (if stale) and return the path of librfi.so (or of librfi_debug.so)."""
    lib = DEBUG_LIB if debug_bounds else LIB
    if not force and os.path.exists(lib):
        newest = max(os.path.getmtime(f) for f in _inputs())
        if os.path.getmtime(lib) >= newest:
            return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    objdir = os.path.join(HERE, "_lib", "obj_debug" if debug_bounds else "obj")
    os.makedirs(objdir, exist_ok=True)
    extra = ["-DRFI_DEBUG_BOUNDS"] if debug_bounds else []
    # translation units compile in parallel, then one link step
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", f".{os.getpid()}.o"))
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append(subprocess.Popen(cmd))
        objs.append(obj)
    failed = [p.wait() for p in procs]
    if any(failed):
        raise RuntimeError(f"nvcc failed for {[s for s, r in zip(SOURCES, failed) if r]}")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "--cudart", "static", "-shared", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
