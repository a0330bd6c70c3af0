"""Seeded synthetic inputs for the boundary-integral Poisson-Boltzmann path.

This package is shared by the CPU oracle side (tests, the oracle timing leg of
``bench.py``) and the CUDA side (tests, ``bench.py``).  It builds geometry and
charges only: triangulated spheres and radially displaced spheres, their
per-triangle centroid / unit normal / area, and point charges inside them.
It contains none of the solver's arithmetic (no Green's functions, no kernels,
no sums over pairs), so neither side borrows the other's mathematics from it.

The paper meshes real proteins with MSMS (Sec. 2.1 and Sec. 3); those
structures are not available here, so these seeded surfaces stand in for them
with the same element counts, element sizes and charge densities.
"""
from .surfaces import (  # noqa: F401
    icosphere,
    displaced_icosphere,
    triangle_geometry,
    real_sph_harm_sum,
    charges_in_ball,
    charges_inside_surface,
    Problem,
    born_problem,
    kirkwood_problem,
    protein_like_problem,
    batched_charges,
    uneven_batch_problems,
    adjoint_problem,
    two_spheres_problem,
    strongly_displaced_problem,
    problem_by_name,
    PROBLEM_NAMES,
)
