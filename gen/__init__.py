"""Seeded synthetic inputs for the GenEO hot path.

This module only builds *inputs*: structured Q1 meshes, element stiffness
matrices of the Darcy problem (Section 2, eq. 2) and of linear elasticity
(Section 2, eq. 3), coefficient fields, the assembled global matrix with the
Dirichlet rows and columns eliminated, the load vector and a box partition
into overlapping subdomains (Section 3, first paragraphs).  It holds none of
the preconditioner's arithmetic (partition of unity, local matrices, eigen
problems, coarse space, solver); those live separately in the oracle and in
the CUDA library, which both consume the arrays produced here.
"""
from .problems import (  # noqa: F401
    Problem,
    q1_reference_stiffness,
    q1_reference_load,
    q1_elasticity_element,
    orthotropic_stiffness,
    isotropic_stiffness,
    structured_mesh,
    box_partition,
    darcy_problem,
    uneven_darcy_problem,
    kd_partition,
    elasticity_problem,
    kappa_channels_2d,
    kappa_skyscrapers_2d,
    kappa_layers_2d,
    kappa_grf_layers_3d,
    gaussian_random_field,
    splitmix64,
)
