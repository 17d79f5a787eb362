"""Seeded synthetic image generators shared by the tests, the benchmark and
the oracle checks.  They hold none of the codec's arithmetic: they only make
uint8 planes (and per-image parameters) from a seed."""
from .images import (  # noqa: F401
    sinusoid_image,
    powerlaw_image,
    yuv420_frame,
    batch_workload,
    ratecontrol_workload,
    stream_workload,
    ragged_sizes,
)
