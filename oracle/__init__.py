"""FP64 CPU oracle for the D3Q19 cascaded LBM (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package. The GPU library never does.
"""
from .oracle import (  # noqa: F401
    Lattice, build, lib_path, velocities, moment_exponents, matrix_M, matrix_Minv,
    matrix_N, matrix_S, teq, cforce, central_moments, macros_node, collide,
    equilibrium, init, step, step_decay, macros, first_step_nodes, adjoint_step, adjoint_seed,
    num_threads, feq_discrete, guo_force,
)
