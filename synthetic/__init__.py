"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only draws random numbers and shapes density fields; it holds none of the
homogenization method's arithmetic (no stiffness, no solve, no filter, no update).
Every generator is a pure function of its arguments (seed included), built on one
counter-based generator (splitmix64 of seed and element index), so the CUDA side and
the oracle always see bit-identical inputs within a process.
"""
from .generators import (  # noqa: F401
    splitmix64_uniform,
    uniform_density,
    uniform_field,
    normal_field,
    conv_net_parameters,
    smoothed_threshold_density,
    sphere_inclusion_density,
    laminate_density,
    cubic_symmetric_density,
    batched_cell_specs,
)
