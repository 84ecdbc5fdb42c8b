"""CPU FP64 oracle for graph-partitioned SP2 (G-SP2).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the CUDA
path is checked against.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference legs may import it; the library itself never does, and the
two share no code.  See ``oracle/gsp2.py`` for the functions and the passages of
the paper each one follows.
"""

from .gsp2 import (  # noqa: F401
    gershgorin_bounds,
    initial_guess,
    sp2_step,
    branch_alpha,
    sp2_dense,
    core_halo,
    ch_cost,
    stop_now,
    tail_alpha,
    gsp2,
    gsp2_tail,
    GSP2Result,
    eig_projector,
    sp2_map_on_spectrum,
    gsp2_adjoint,
    part_adjoint,
    seed_on_pattern,
    dk_adjoint,
    fd_directional,
)
