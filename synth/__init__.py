"""Seeded synthetic ptychography inputs shared by the oracle tests, the GPU tests and the bench.

This package simulates the *measurement* only (object, probe, scan, detector
intensities with partial coherence and Poisson noise). It hands both the FP64
oracle and the CUDA path plain arrays and computes nothing that the
reconstruction engine itself computes (no twiddles, no blur kernels of the
engine, no modulus ratios).
"""
from .generators import (  # noqa: F401
    Problem,
    make_problem,
    far_field_object_pixel,
    qpt_phase,
    electron_wavelength,
    CONFIG_NAMES,
)
