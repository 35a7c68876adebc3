"""Oracle: the absorption spectrum eps_2(omega) (steps A7, A8).

Test infrastructure only (see package docstring).

Eq. epsilon_chi_bar with the TDA (N = identity, Appendix A) and f_S = 1 for
e-h pairs gives, with P the conjugated k.p pair density divided by |q|,

    eps_2(w) = -C Im[ P^H (z - H)^{-1} P ],  z = w + i eta,  C = 8 pi / (Omega Nk)

(2 for spin, 1/Nk from the Bloch normalisation).  Two evaluations:

- ``eps2_dense``: the paper's route, eigenpairs of H (Eqs. bse_eig, resolvent):
  eps_2 = C sum_l |P^H A_l|^2 eta / ((w - E_l)^2 + eta^2).
- ``haydock`` + ``continued_fraction``: Lanczos from v_0 = P/|P| on H with
  classical Gram-Schmidt applied twice against the whole basis at every step,
  a_j = Re(v_j^H H v_j) (accumulated over both passes), b_{j+1} = |w|; the
  spectrum is -C |P|^2 Im g(z) with g(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ...)),
  no terminator.  Breakdown: b_{j+1} <= 1e-10 |H v_j| stops the recursion (the
  Krylov space is invariant, so the truncated fraction is exact).

``ritz``: eigenvalues and first-component weights of the tridiagonal (the pole
expansion of g), i.e. exciton energies and normalised oscillator strengths.

Pinned by tests/test_oracle_spectrum.py: dense == Haydock(N = dim) to 1e-10,
kernel-off closed form, moment identities, rigid scissor shift; the Ritz pairs
against the dense eigenvalues of T, their moments, the pole expansion of the
continued fraction, and the eigenpairs of H at full Krylov dimension.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import geometry as geo

PI = 3.141592653589793
BREAKDOWN_REL = 1e-10


def prefactor(spec) -> float:
    return 8.0 * PI / (geo.cell_volume(spec) * spec.nkpt)


def eps2_dense(spec, H, P, omega, eta) -> np.ndarray:
    e, a = scipy.linalg.eigh(H)
    wts = np.abs(np.conj(P) @ a) ** 2
    d = omega[:, None] - e[None, :]
    return prefactor(spec) * (eta / (d * d + eta * eta)) @ wts


def eps2_independent(spec, de, P, omega, eta) -> np.ndarray:
    """Kernel off: H diagonal, eps_2 = C sum_S |P_S|^2 eta/((w - de_S)^2 + eta^2)."""
    d = omega[:, None] - de[None, :]
    return prefactor(spec) * (eta / (d * d + eta * eta)) @ (np.abs(P) ** 2)


def haydock(H, P, nsteps):
    """Returns (a [n], b [n], steps_done, V [n][dim]); b[0] = 0, b[j] couples j-1 and j."""
    dim = len(P)
    nsteps = min(nsteps, dim)
    V = np.zeros((nsteps, dim), dtype=np.complex128)
    a = np.zeros(nsteps)
    b = np.zeros(nsteps)
    v = P / np.linalg.norm(P)
    done = nsteps
    for j in range(nsteps):
        V[j] = v
        w = H @ v
        scale = np.linalg.norm(w)
        basis = V[: j + 1]
        h1 = np.conj(basis) @ w
        w = w - basis.T @ h1
        h2 = np.conj(basis) @ w
        w = w - basis.T @ h2
        a[j] = (h1[j] + h2[j]).real
        bn = np.linalg.norm(w)
        if j + 1 < nsteps:
            if bn <= BREAKDOWN_REL * scale:
                done = j + 1
                break
            b[j + 1] = bn
            v = w / bn
    return a[:done], b[:done], done, V[:done]


def continued_fraction(a, b, z) -> np.ndarray:
    """g(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ... - b_{n-1}^2/(z - a_{n-1}))), from the bottom up."""
    z = np.asarray(z, dtype=np.complex128)
    g = np.zeros_like(z)
    n = len(a)
    for j in range(n - 1, -1, -1):
        tail = b[j + 1] ** 2 * g if j + 1 < n else 0.0
        g = 1.0 / (z - a[j] - tail)
    return g


def eps2_haydock(spec, H, P, omega, eta, nsteps):
    a, b, done, _ = haydock(H, P, nsteps)
    g = continued_fraction(a, b, omega + 1j * eta)
    return -prefactor(spec) * np.vdot(P, P).real * g.imag, a, b, done


def ritz(a, b):
    """Eigenvalues theta_i (ascending) and weights w_i = (first eigenvector component)^2 of the Lanczos
    tridiagonal T (diagonal a, off-diagonal b[1:]): the poles and residues of g(z) = sum_i w_i/(z - theta_i),
    i.e. exciton energies and normalised oscillator strengths |P^H A_l|^2/|P|^2 of the converged states."""
    n = len(a)
    if n == 1:
        return np.array([a[0]]), np.array([1.0])
    th, y = scipy.linalg.eigh_tridiagonal(np.asarray(a, dtype=np.float64), np.asarray(b[1:n], dtype=np.float64))
    return th, y[0, :] ** 2
