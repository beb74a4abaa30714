"""Seeded synthetic stereo pairs shared by the oracle tests, the GPU tests and the bench.

This package holds no part of the matching method's arithmetic: it only draws images,
disparity maps and request streams from seeded random generators.
"""

from .stereo import (  # noqa: F401
    StereoPair,
    blurred_noise,
    make_pair,
    config_pair,
    batch_specs,
    serving_requests,
)
