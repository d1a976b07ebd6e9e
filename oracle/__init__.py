"""FP64 CPU oracle for the online RFI flagging path (arXiv 2412.14775).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
bench's CPU-baseline leg, never by the product path.  It shares no code with the
CUDA library.  Parity is pinned by the closed forms and invariants in
tests/test_oracle_pins.py (SK null mean and variance, Cauchy-Schwarz bounds,
fully polarised tone, isotropic null, Hermitian autocorrelations, averaging by
brute force, exact small-grid evaluation, block-split invariance, footprints,
partial windows, online thresholds, overlapping windows).
"""
from .adaptive import AdaptiveOracleStream
from .sliding import SlidingOracleStream
from .oracle import (OracleStream, outputs_for, stokes, sk_window, ds_window, flag,
                     to_f64_rows)

__all__ = ["AdaptiveOracleStream", "OracleStream", "SlidingOracleStream", "outputs_for",
           "stokes", "sk_window", "ds_window", "flag", "to_f64_rows"]
