"""Plain FP64 CPU oracle of the GenEO two-level Schwarz method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it shares no code with the CUDA library: both consume the
same seeded inputs from ``gen`` and nothing else.
"""
from .geneo_oracle import (  # noqa: F401
    OracleOptions,
    GenEOOracle,
    subdomain_sets,
    element_multiplicity,
    partition_of_unity,
    sarkis_partition_of_unity,
    dirichlet_matrix,
    neumann_matrix,
    overlap_matrix,
    geneo_pencil,
    local_eigenpairs,
    select_count,
    coarse_vectors,
    coarse_matrix,
    pcg,
    lanczos_condition_estimate,
    theorem1_bound,
)
