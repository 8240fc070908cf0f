"""Seeded synthetic inputs shared by the oracle-side tests, the GPU tests and the benchmark.

This package holds no arithmetic of the eigensolver itself: it only builds the
sparse operators, the diagonal metric B, the potentials and the random blocks
(X0, the Gaussian sketch Omega of the norm estimate, the gradient probes g_i)
from a seed.  Random numbers come from one counter-based generator,
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), so any consumer can regenerate any element from
(seed, stream, index) alone.
"""
from .philox import (philox4x32_10, uniform52, normal_flat, normal_block, uniform_block,
                     STREAM_X0, STREAM_BDIAG, STREAM_COEF, STREAM_POTENTIAL,
                     STREAM_OMEGA, STREAM_GRAD)
from .problems import (CSR, Problem, laplacian_1d, laplacian_2d_dirichlet,
                       laplacian_3d_dirichlet, diffusion_3d_lognormal,
                       hamiltonian_3d_periodic, tridiag, add_diagonal, mass_matrix_2d,
                       closed_form_mass_pencil,
                       block_width, make_problem, WORKLOADS)

__all__ = [
    "philox4x32_10", "uniform52", "normal_flat", "normal_block", "uniform_block",
    "STREAM_X0", "STREAM_BDIAG", "STREAM_COEF", "STREAM_POTENTIAL",
    "STREAM_OMEGA", "STREAM_GRAD",
    "CSR", "Problem", "laplacian_1d", "laplacian_2d_dirichlet",
    "laplacian_3d_dirichlet", "diffusion_3d_lognormal",
    "hamiltonian_3d_periodic", "tridiag", "add_diagonal", "mass_matrix_2d",
    "closed_form_mass_pencil", "block_width",
    "make_problem", "WORKLOADS",
]
