"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds no arithmetic of the traversability method: it only draws elevation
maps, poses and shift sequences from numpy's ``default_rng``.  Both the CUDA path and
the CPU oracle are fed the very same arrays produced here.
"""
from .terrain import (  # noqa: F401
    bumpy_plane,
    fractal_steps_nan,
    fractal_world,
    lidar_scan,
    lookup_poses,
    obstacle_risk,
    random_se2_grid,
    shift_sequence,
    random_poses,
    tilted_plane,
)
