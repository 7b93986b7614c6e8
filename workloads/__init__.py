"""Seeded synthetic inputs for the FEAST interval eigensolver.

This package builds test and benchmark inputs only: planted-spectrum Hermitian
matrices A = Q diag(lambda) Q^H and random starting subspaces.  It holds none of
the eigensolver's arithmetic, so both the CPU oracle and the CUDA path can take
their inputs from it without sharing any method code.
"""
from .planted import (  # noqa: F401
    Problem,
    planted_matrix,
    planted_general,
    haar_unitary,
    random_subspace,
    spectrum_config1,
    spectrum_config2,
    spectrum_config3,
    spectrum_config4,
    spectrum_config5,
    spectrum_disk,
    spectrum_paper,
    spectrum_dense_edge,
    spectrum_uniform,
    make_problem,
)
