"""Seeded synthetic inputs for the LRBMS two-phase online step.

This package only draws random numbers and lays out problem data (grids,
permeability and porosity fields, boundary tags, training parameters, basis
sizes, random rotations). It holds none of the method's arithmetic: no
discretisation, no projection, no solve. Both the CPU oracle (in tests) and the
GPU library consume what it returns.

The paper's benchmark fields exist only as figures, so every workload here is
a seeded stand-in with the shapes and value distributions of the workloads
listed in ``synth.problems``.
"""
from .fields import lognormal_field, layered_lognormal_field  # noqa: F401
from .problems import (  # noqa: F401
    Problem,
    make_problem,
    simplex_params,
    basis_sizes,
    random_orthogonal,
    boundary_face_count,
)
