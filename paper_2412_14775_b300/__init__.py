"""B300 (sm_103a) online RFI flagging: spectral kurtosis plus polarisation
directional statistics over windows, flags, and flagged averaging
(arXiv 2412.14775, Sections 2-2.2).

The computation lives in the CUDA library librfi.so behind the C ABI of
include/rfi.h; `binding` exposes those entry points under the same names.
"""
from . import binding
from .binding import RfiError
from .stream import RfiStream
from .thresholds import default_thresholds

__all__ = ["binding", "RfiError", "RfiStream", "default_thresholds"]
