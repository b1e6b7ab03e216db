"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package holds problem set-ups only: block meshes (lists of leaf blocks), initial
conditions written as closed-form functions of the cell centres, and the SplitMix64
counter generator used for noise and random Fourier phases.  It contains none of the
numerical method (no fluxes, limiters, ghost filling, time steps); neither the oracle
nor the CUDA path is imported here.
"""

from .mesh import Mesh, Problem, uniform_mesh, radial_amr_mesh, slab_amr_mesh, ensemble_mesh
from .problems import (
    NVAR, VAR_NAMES, conserved_from_primitive, cell_centres, evaluate_on_mesh,
    orszag_tang, alfven_wave, rotor, harris_sheet, ensemble_problem, advection_2d,
    brio_wu, field_loop, uniform_state, blast_wave, divb_bump, CONFIGS,
)

__all__ = [
    "Mesh", "Problem", "uniform_mesh", "radial_amr_mesh", "slab_amr_mesh", "ensemble_mesh",
    "NVAR", "VAR_NAMES", "conserved_from_primitive", "cell_centres", "evaluate_on_mesh",
    "orszag_tang", "alfven_wave", "rotor", "harris_sheet", "ensemble_problem",
    "advection_2d", "brio_wu", "field_loop", "uniform_state", "blast_wave", "divb_bump",
    "CONFIGS",
]
