"""The debug-bounds build (every global access of the kernels checked against the
extent its launch declares; a violation is skipped and reported by rfi_check) runs the
GPU parity, batching, partial-window, online-threshold, launch-overlap (including
independent launches) and random-combination tests.
They must pass unchanged: the checks alter no result, and no kernel touches memory
outside its buffers on any of those shapes.

compute-sanitizer is not available on the GPU pool; this build stands in for its
memory checker.  Each parity stream ends with rfi_check, which fails on any caught
access."""
import os
import subprocess
import sys

import pytest

from paper_2412_14775_b300 import build as lib_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_debug_bounds_build():
    lib = lib_build.build(debug_bounds=True)          # compiles only if missing or stale
    env = dict(os.environ, RFI_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_parity_gpu.py", "tests/test_adaptive_gpu.py", "tests/test_fuzz_gpu.py",
           "tests/test_sliding_gpu.py", "tests/test_overlap_gpu.py", "tests/test_wpar_gpu.py",
           "-k", "shapes or partial or batch or host or tma or buffered or footprints or "
                 "checkpoint or degenerate or online or warm_up or edge or random or "
                 "sliding or overlap or independent or window_parallel"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail


def test_debug_build_is_the_library_loaded():
    """The subprocess above really loads the checked build."""
    lib = lib_build.build(debug_bounds=True)
    code = ("import paper_2412_14775_b300.binding as B, ctypes; B.load_library(); "
            "print(B.LIB_PATH)")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, RFI_LIBRARY=lib), timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == lib
