"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package builds the finite-element stiffness/mass pencils (A, B) and the
random start blocks that the rational-filter subspace iteration consumes.  It
holds none of the eigensolver's arithmetic: no filter, no shifted solve, no
Rayleigh-Ritz.  Everything is deterministic in its seed.
"""
from .fe import (Pencil, pencil_1d, pencil_2d_q1, pencil_3d_elasticity, rigid_body_modes,
                 start_block, config_pencil, CONFIGS, interval_for, weyl_gamma,
                 random_problem, batch_workload, serving_stream)

__all__ = ["Pencil", "pencil_1d", "pencil_2d_q1", "pencil_3d_elasticity", "rigid_body_modes",
           "start_block", "config_pencil", "CONFIGS", "interval_for", "weyl_gamma",
           "random_problem", "batch_workload", "serving_stream"]
