"""FP64 CPU oracle of the pc-engine (test infrastructure; see pc_engine.py)."""
from .pc_engine import (  # noqa: F401
    Params,
    gaussian_kernel,
    blur,
    fresnel_tf,
    propagate_forward,
    propagate_backward,
    modulus,
    cbar_per_position,
    complex_constraint,
    default_eps,
    in_window,
    iteration,
    iterate,
)
