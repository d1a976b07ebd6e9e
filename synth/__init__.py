"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

Holds none of the flagging method's arithmetic."""
from .generate import (n_baselines, baseline_pairs, tiny_block, lofar_block,
                       serving_streams, BATCH_STATIONS, BATCH_CHANNELS)

__all__ = ["n_baselines", "baseline_pairs", "tiny_block", "lofar_block", "serving_streams",
           "BATCH_STATIONS", "BATCH_CHANNELS"]
