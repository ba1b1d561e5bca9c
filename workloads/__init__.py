"""Seeded synthetic inputs for the infinite-cell Clenshaw-Curtis SQ sweep.

This package only draws atom positions and samples the fixed effective potential
V_eff on the grid. It contains none of the method's arithmetic, so both the CPU
oracle and the CUDA library may take their inputs from it.
"""
from .sq_workloads import (  # noqa: F401
    CONFIGS,
    make_instance,
    make_batch,
    make_profile_case,
    tiny_instance,
    gaussian_veff,
    random_positions,
    perturb_positions,
)
