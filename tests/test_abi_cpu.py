"""The C ABI library without a GPU: it loads, exports every symbol include/rfi.h
declares, the Python binding uses the same names, and calls fail cleanly."""
import ctypes
import os
import re

import pytest

from paper_2412_14775_b300 import binding, build, default_thresholds
from paper_2412_14775_b300.thresholds import sk_sigma

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "rfi.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(rfi_\w+)\s*\(", text, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    names = _declared()
    assert len(names) >= 16, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names():
    assert sorted(binding.EXPORTED) == _declared()
    for n in binding.EXPORTED:
        assert callable(getattr(binding, n))


def test_status_strings():
    assert binding.rfi_status_str(0) == "RFI_OK"
    for s in range(1, 7):
        assert binding.rfi_status_str(s).startswith(binding.STATUS[s])
    assert "unknown" in binding.rfi_status_str(99)


def test_calls_fail_cleanly_without_device():
    lib = binding.load_library()
    assert lib.rfi_destroy(None) == 0
    assert lib.rfi_process_block(None, None, 16, None, None, None, None, None) == 1
    assert lib.rfi_reset(None) == 5
    n = ctypes.c_int()
    assert lib.rfi_outputs_for(None, 16, ctypes.byref(n)) == 5
    h = ctypes.c_void_p()
    t = binding.rfi_thresholds(1.0, 0.5, 2.0, 0.5, 2 ** -23)
    # argument errors are reported before any CUDA call
    assert lib.rfi_create(ctypes.byref(h), 0, 4, 16, 64, ctypes.byref(t), 0) == 1
    assert lib.rfi_create(ctypes.byref(h), 4, 4, 1, 64, ctypes.byref(t), 0) == 1
    assert lib.rfi_create(ctypes.byref(h), 4, 4, 16, 40, ctypes.byref(t), 0) == 1
    bad = binding.rfi_thresholds(1.0, 2.0, 0.5, 0.5, 2 ** -23)
    assert lib.rfi_create(ctypes.byref(h), 4, 4, 16, 64, ctypes.byref(bad), 0) == 1
    nan = binding.rfi_thresholds(float("nan"), 0.5, 2.0, 0.5, 2 ** -23)
    assert lib.rfi_create(ctypes.byref(h), 4, 4, 16, 64, ctypes.byref(nan), 0) == 1
    assert h.value is None
    assert b"K=40" in lib.rfi_last_error() or lib.rfi_last_error()
    with pytest.raises(binding.RfiError):
        binding.rfi_create(4, 4, 16, 64, default_thresholds(16), "f32")  # no GPU here


def test_default_thresholds():
    t = default_thresholds(16)
    assert t["s_low"] < 1.0 < t["s_high"]
    assert abs(t["gamma"] - (7.814727903251178 / 48) ** 0.5) < 0.01 * t["gamma"]   # chi2(3) limit
    # d = 1 reduces to the classic SK variance 4 M^2 / ((M-1)(M+2)(M+3))
    for M in (8, 16, 64):
        assert abs(sk_sigma(M, 1.0) ** 2 - 4 * M * M / ((M - 1) * (M + 2) * (M + 3))) < 1e-14


def test_header_is_c_and_matches_the_binding(tmp_path):
    """include/rfi.h compiles as strict C99 against librfi.so, calls fail cleanly from C
    without a GPU, and the structures have the sizes and field offsets the ctypes
    binding assumes."""
    import os
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = build.build()
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "abi.c"
    src.write_text(r"""
#include <stddef.h>
#include <stdio.h>
#include "rfi.h"
int main(void) {
    rfi_ctx *ctx = (rfi_ctx *)1;
    rfi_thresholds thr = {1.0, 0.0, 2.0, 0.5, 1e-7};
    int rc = rfi_create(NULL, 4, 4, 16, 64, &thr, RFI_C64);
    printf("%d %d %s\n", rc, ctx != NULL, rfi_status_str(RFI_EINVAL));
    printf("%zu %zu %zu\n", sizeof(rfi_options), sizeof(rfi_thresholds), sizeof(rfi_adaptation));
    printf("%zu %zu %zu\n", offsetof(rfi_options, partial_windows),
           offsetof(rfi_options, adaptive), offsetof(rfi_adaptation, n_warm));
    return 0;
}
""")
    exe = tmp_path / "abi"
    subprocess.check_call([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", inc,
                           str(src), "-o", str(exe), lib, f"-Wl,-rpath,{os.path.dirname(lib)}"])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    rc, _, name = out[0].split(" ", 2)
    assert int(rc) == 1 and name.startswith("RFI_EINVAL")
    sizes = [int(x) for x in out[1].split()]
    assert sizes == [ctypes.sizeof(binding.rfi_options), ctypes.sizeof(binding.rfi_thresholds),
                     ctypes.sizeof(binding.rfi_adaptation)]
    offs = [int(x) for x in out[2].split()]
    assert offs == [binding.rfi_options.partial_windows.offset, binding.rfi_options.adaptive.offset,
                    binding.rfi_adaptation.n_warm.offset]
