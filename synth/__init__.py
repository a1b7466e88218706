"""Seeded synthetic inputs (point clouds and right-hand sides).

This module holds only input generation: it contains none of the solver's
arithmetic, so both the CUDA path and the CPU oracle may draw their inputs
from it.  Every generator takes an explicit seed and uses numpy's PCG64
``default_rng``, so the same call returns the same points on any machine.

The point sets stand in for the paper's workloads: a uniform unit cube with
the Laplace kernel (Section IV) and surface point clouds of a complex
geometry with the Yukawa kernel (Section V).  The paper's hemoglobin BEM
mesh is not available, so a union of ellipsoid and torus surfaces replaces
it.
"""
from .points import (cube, line, sphere_ball, surface_union, batched_problems,
                     cube_surface, sphere_surface, ellipsoid_surface, rhs,
                     workload)

__all__ = ["cube", "line", "sphere_ball", "surface_union", "batched_problems",
           "cube_surface", "sphere_surface", "ellipsoid_surface", "rhs",
           "workload"]
