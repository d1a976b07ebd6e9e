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
           "rfi_inst_wp_f32.cu", "rfi_inst_wp_f16.cu", "rfi_inst_h2.cu"]
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
    """Compile (if stale) and return the path of librfi.so (or of librfi_debug.so).

    Objects are kept per build flavour; a translation unit is recompiled when it, or
    any header of the library, is newer than its object."""
    lib = DEBUG_LIB if debug_bounds else LIB
    headers = [f for f in _inputs() if not f.endswith(".cu")]
    newest_header = max(os.path.getmtime(f) for f in headers)
    objdir = os.path.join(HERE, "_lib", "obj_debug" if debug_bounds else "obj")
    objs = [os.path.join(objdir, src.replace(".cu", ".o")) for src in SOURCES]

    def fresh(src, obj):
        return (os.path.exists(obj) and os.path.getmtime(obj) >=
                max(os.path.getmtime(os.path.join(CSRC, src)), newest_header))

    # up to date: every object newer than its sources (a source edited while an earlier
    # build ran leaves its object stale) and the library newer than every object
    if (not force and os.path.exists(lib) and all(fresh(s, o) for s, o in zip(SOURCES, objs))
            and os.path.getmtime(lib) >= max(os.path.getmtime(o) for o in objs)):
        return lib
    os.makedirs(os.path.dirname(lib), exist_ok=True)
    os.makedirs(objdir, exist_ok=True)
    extra = ["-DRFI_DEBUG_BOUNDS"] if debug_bounds else []
    # stale translation units compile in parallel, then one link step
    procs, tmps = [], []
    for src, obj in zip(SOURCES, objs):
        path = os.path.join(CSRC, src)
        if not force and not verbose and fresh(src, obj):
            continue
        tmp = obj + f".tmp{os.getpid()}"
        cmd = [NVCC, *ARCH, *FLAGS, *extra, "-c", "-o", tmp, path]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd)))
        tmps.append((tmp, obj))
    failed = [src for src, p in procs if p.wait()]
    if failed:
        for tmp, _ in tmps:
            if os.path.exists(tmp):
                os.remove(tmp)
        raise RuntimeError(f"nvcc failed for {failed}")
    for tmp, obj in tmps:
        os.replace(tmp, obj)
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([NVCC, *ARCH, "--cudart", "static", "-shared", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, debug_bounds="--debug-bounds" in sys.argv))
