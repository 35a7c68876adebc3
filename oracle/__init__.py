"""CPU oracle for the plane-wave Bethe-Salpeter hot path (TEST INFRASTRUCTURE).

A plain, slow, complex128 numpy/scipy restatement of what the paper defines:
pair densities (Eq. pair_density), the e-h exchange and screened direct kernels
(Eqs. V_eh, W_SS), the Tamm-Dancoff Hamiltonian (Eq. kernel, Sec. II C), the
k.p dipole (Eq. density_matrix), the spectrum from the spectral representation
of the irreducible response (Eq. epsilon_chi_bar, Appendix A), its gradient, the static
RPA screening from the independent-particle response (Eqs. chi0_GG, epsilon_-1), the problem
with e-h / h-e coupling beyond the Tamm-Dancoff approximation (Appendix A), and the q-point
symmetry reduction of W (Sec. III A), and the macroscopic dielectric function from TDDFT with
local fields (Sec. II A-B).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1206_3518_gb300``) and neither imports the other; both read inputs
from ``synth``.

Parity status per function is stated in each module header; every function is
pinned by ``tests/test_oracle_*.py`` against closed forms, brute force,
invariants or textbook limits.
"""
from . import geometry, pair, kernel, spectrum, adjoint, screening, coupling, symmetry, tddft  # noqa: F401
