"""Seeded synthetic inputs for the plane-wave BSE hot path.

This package is the single source of inputs for both the CUDA path and the
CPU oracle.  It draws random numbers and shapes them into physically plausible
inputs (orthonormal plane-wave coefficients, band energies, a model statically
screened interaction W_GG'(q)); it holds none of the method's own arithmetic
(pair densities, kernels, Hamiltonian, spectrum).
"""
from .systems import (  # noqa: F401
    HARTREE_EV,
    SystemSpec,
    BulkSystem,
    config_spec,
    generate,
    generate_slab_batch,
    slab_batch_specs,
    omega_grid,
)
