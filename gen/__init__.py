"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This package draws random numbers and lays them out as arrays; it holds none
of the boundary-element arithmetic (no kernels, no panel integrals, no
solves).  Everything the method itself computes is done separately by the
oracle and by the CUDA library.
"""
from .scenes import (  # noqa: F401
    CONFIGS,
    Scene,
    make_scene,
    make_samples,
    analytic_truth,
    add_noise,
    perturb,
    batch_scenes,
    crossing_fraction,
    SEGMENT_CONFIGS,
    SegmentScene,
    make_segment_scene,
)
