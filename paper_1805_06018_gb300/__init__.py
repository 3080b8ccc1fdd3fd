"""GB300-native product-convolution apply (arXiv 1805.06018, Section 3.2).

The compute lives in libpc.so (CUDA for sm_103a, C ABI in include/pc.h);
:mod:`.binding` marshals arguments to it.  There is no CPU or library
fallback: if libpc.so is missing every entry point raises LibraryMissing.
"""
from .binding import (BlockPlan, Context, Estimator, LibraryMissing, Operator, PCError, Server, lib, pc_autotune,  # noqa: F401
                      pc_extend_impulse, pc_harmonic_weights, pc_neighbourhood_boxes, pc_sample_points)

__all__ = ["Context", "Operator", "BlockPlan", "Estimator", "Server", "PCError", "LibraryMissing", "lib", "pc_autotune", "pc_sample_points",
           "pc_neighbourhood_boxes", "pc_harmonic_weights", "pc_extend_impulse"]
