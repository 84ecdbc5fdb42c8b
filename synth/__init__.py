"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only produces input data (a tight-binding Hamiltonian in CSR form, a
partition of its orbitals and the dependency graph that defines halos).  It holds
none of the density-matrix method's arithmetic: no spectral bounds, no purification,
no halo construction and no scatter/gather.
"""

from .tb import (  # noqa: F401
    TBSystem,
    WORKLOADS,
    make_tb_system,
    make_workload,
    rcb_partition,
    block_partition,
    locality_graph,
    dense_from_csr,
    csr_from_dense,
    random_symmetric_on_pattern,
)
