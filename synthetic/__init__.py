"""Seeded synthetic robust-planning problems.

This package only builds problem instances (voxel grid, structures, proton
spots, per-scenario dose-influence matrices in CSR form).  It contains none of
the optimisation method's arithmetic, so both the CPU oracle and the CUDA
library can be fed from it without sharing any solver code.
"""
from .phantom import (  # noqa: F401
    Problem,
    config_tiny_plain,
    from_dense,
    config_realistic,
    random_problem,
    scenario_set_13,
    scenario_set_49,
    reweighted,
    block_diagonal,
    config_batch,
    BATCH_SIZES_SMALL,
    sample_weights,
    N_WEIGHT_SLOTS,
)
