"""Oracle: macroscopic dielectric function from TDDFT with local fields (Sec. II A-B).

Test infrastructure only (see package docstring).

Definitions followed, in the optical limit q -> 0 along qhat, on the q = 0 sphere of the system:

- Adler-Wiser response (Eq. chi0_GG) with the occupied bands v and empty bands c of the system:
  v -> c terms (f_v - f_c = 1) and c -> v terms (f_c - f_v = -1), spin 2, k sum normalised over the
  Born-von Karman supercell (1/(Omega Nk)), transition energies e_c + Delta - e_v (Delta the scissor
  shift of step A5; Delta = 0 gives the Kohn-Sham energies).  In the symmetrised form
  chi~0 = v^1/2 chi0 v^1/2 (v^1/2(q + G) = sqrt(4 pi)/|q + G|):

      chi~0_GG'(w) = 2/(Omega Nk) sum_S [ a_S(G) conj(a_S(G')) / (w - de_S + i eta)
                                         - abar_S(G) conj(abar_S(G')) / (w + de_S + i eta) ],

  a_S(G) = v^1/2(G) rho_vc^{kk}(G), abar_S(G) = v^1/2(G) rho_cv^{kk}(G) = v^1/2(G) conj(rho_vc^{kk}(-G))
  for G != 0 (Eq. pair_density at q = 0), and at G = 0 the k.p limit of Eq. density_matrix:
  v^1/2(q) rho_vc^{k,k+q}(0) -> sqrt(4 pi) conj(P_S) and v^1/2(q) rho_cv^{k,k+q}(0) -> -sqrt(4 pi) P_S,
  P_S the dipole of step A6.
- Dyson equation (Eq. Dyson_GG) with the kernel K = v + f_xc (RPA: f_xc = 0; ALDA: the local-density
  xc kernel below), symmetrised: chi~ = chi~0 + chi~0 (I + F) chi~, F = v^-1/2 f_xc v^-1/2.
- Eq. epsilon_-1: eps^-1 = I + chi~, and Eq. epsilon_M: eps_M(w) = 1/[eps^-1]_00.  Without local
  fields (only G = 0 kept) eps_M = 1 - chi~0_00.
- ALDA: f_xc(r) = d^2(n eps_xc)/dn^2 at the ground-state density n(r) = 2/(Omega Nk) sum_{k,v} |u_vk(r)|^2
  (u the unnormalised inverse transform of step A1), eps_xc = Slater exchange + the Perdew-Zunger
  parametrisation of the Ceperley-Alder correlation energy (spin-unpolarised), evaluated at
  max(n, n_floor) with n_floor = 1e-6 bohr^-3; f_xc(G, G') = (1/N_r) sum_r f_xc(r) exp(-i(G - G').r) on the
  real-space grid, and F_GG' = |G| f_xc(G, G') |G'|/(4 pi) (zero row and column at G = 0 for q -> 0).

Pinned by tests/test_oracle_tddft.py: without local fields Im eps_M equals the independent-particle
eps_2 of step A8 minus its mirror at -w (closed form); with RPA local fields eps_M equals 1 minus the
response of the full Bethe-Salpeter problem with the exchange kernel alone (Appendix A, the coupled
form of coupling.py), and with ALDA local fields the same problem with the xc kernel added to the
exchange; the density integrates to 2 Nv electrons per cell; the xc kernel equals the numerical second
derivative of n eps_xc; the Perdew-Zunger branches meet at rs = 1 in value and slope; a uniform density
gives a diagonal F.
"""
from __future__ import annotations

import numpy as np

from . import coupling
from . import geometry as geo
from . import kernel as ok
from . import pair

PI = 3.141592653589793
N_FLOOR = 1e-6

# Perdew-Zunger (1981) fit of the Ceperley-Alder correlation energy, spin-unpolarised, Hartree units
PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116


def sqrt_coulomb0(spec) -> np.ndarray:
    """v^1/2(G) = sqrt(4 pi)/|G| on the q = 0 sphere (0 at G = 0: that entry comes from the k.p limit)."""
    g0 = geo.sphere(spec, (0, 0, 0))
    p = geo.cart(spec, (0, 0, 0), g0)
    n = np.sqrt(np.sum(p * p, axis=1))
    out = np.zeros(len(g0))
    out[n > 0] = np.sqrt(4.0 * PI) / n[n > 0]
    return out


def optical_pairs(spec, s, P=None):
    """(a, abar) [dim][NG0]: v^1/2 times the v -> c and c -> v pair densities at q -> 0."""
    rho = pair.exchange_rho(spec, s.gk, s.coef)                   # rho_vc^{kk}(G), S = (k, v, c)
    if P is None:
        P = pair.dipole(spec, s.gk, s.coef, s.energies)
    vs = sqrt_coulomb0(spec)
    mi = coupling.minus_g_index(spec)
    a = rho * vs[None, :]
    abar = np.conj(rho[:, mi]) * vs[None, :]
    a[:, 0] = np.sqrt(4.0 * PI) * np.conj(P)
    abar[:, 0] = -np.sqrt(4.0 * PI) * P
    return a, abar


def chi0_bar(spec, s, omega, eta, delta, P=None) -> np.ndarray:
    """chi~0_GG'(w) [nw][NG0][NG0] (definition above)."""
    a, abar = optical_pairs(spec, s, P)
    de = ok.transition_energies(spec, s.energies, delta)
    pref = 2.0 / (geo.cell_volume(spec) * spec.nkpt)
    out = np.zeros((len(omega), a.shape[1], a.shape[1]), dtype=np.complex128)
    for i, w in enumerate(omega):
        r = 1.0 / (w - de + 1j * eta)
        rb = 1.0 / (w + de + 1j * eta)
        out[i] = pref * ((a.T * r[None, :]) @ np.conj(a) - (abar.T * rb[None, :]) @ np.conj(abar))
    return out


def epsilon_macro(chi0, F=None) -> np.ndarray:
    """eps_M(w) = 1/[eps^-1]_00 with eps^-1 = I + (I - chi~0 (I + F))^-1 chi~0 for every w."""
    n = chi0.shape[1]
    K = np.eye(n) if F is None else np.eye(n) + F
    out = np.zeros(chi0.shape[0], dtype=np.complex128)
    for i in range(chi0.shape[0]):
        x = np.linalg.solve(np.eye(n) - chi0[i] @ K, chi0[i][:, 0])
        out[i] = 1.0 / (1.0 + x[0])
    return out


def epsilon_macro_nlf(chi0) -> np.ndarray:
    """Without local fields: eps_M = 1 - chi~0_00."""
    return 1.0 - chi0[:, 0, 0]


# --- ALDA -----------------------------------------------------------------------------------------------

def realspace_density(spec, s) -> np.ndarray:
    """n(r) [N1][N2][N3] = 2/(Omega Nk) sum_{k,v} |u_vk(r)|^2, u(r) = sum_G c(G) exp(iG.r) (inverse FFT)."""
    n1, n2, n3 = spec.fft
    dens = np.zeros((n1, n2, n3))
    for ik in range(spec.nkpt):
        g = np.asarray(s.gk[ik], dtype=np.int64)
        for iv in range(spec.nv):
            box = np.zeros((n1, n2, n3), dtype=np.complex128)
            box[g[:, 0] % n1, g[:, 1] % n2, g[:, 2] % n3] = s.coef[ik, iv, : len(g)]
            u = np.fft.ifftn(box) * (n1 * n2 * n3)
            dens += np.abs(u) ** 2
    return 2.0 / (geo.cell_volume(spec) * spec.nkpt) * dens


def lda_eps_xc(n):
    """Exchange-correlation energy per electron (Ha) of the uniform gas at density n."""
    n = np.asarray(n, dtype=np.float64)
    ex = -0.75 * (3.0 / PI) ** (1.0 / 3.0) * n ** (1.0 / 3.0)
    rs = (3.0 / (4.0 * PI * n)) ** (1.0 / 3.0)
    hi = PZ_GAMMA / (1.0 + PZ_BETA1 * np.sqrt(rs) + PZ_BETA2 * rs)
    lo = PZ_A * np.log(rs) + PZ_B + PZ_C * rs * np.log(rs) + PZ_D * rs
    return ex + np.where(rs >= 1.0, hi, lo)


def _pz_derivatives(rs):
    """(eps_c, d eps_c/d rs, d^2 eps_c/d rs^2) of the Perdew-Zunger fit."""
    rs = np.asarray(rs, dtype=np.float64)
    sq = np.sqrt(rs)
    D = 1.0 + PZ_BETA1 * sq + PZ_BETA2 * rs
    D1 = PZ_BETA1 / (2.0 * sq) + PZ_BETA2
    D2 = -PZ_BETA1 / (4.0 * rs * sq)
    e_hi = PZ_GAMMA / D
    d1_hi = -PZ_GAMMA * D1 / D ** 2
    d2_hi = -PZ_GAMMA * (D2 / D ** 2 - 2.0 * D1 ** 2 / D ** 3)
    lg = np.log(rs)
    e_lo = PZ_A * lg + PZ_B + PZ_C * rs * lg + PZ_D * rs
    d1_lo = PZ_A / rs + PZ_C * (lg + 1.0) + PZ_D
    d2_lo = -PZ_A / rs ** 2 + PZ_C / rs
    hi = rs >= 1.0
    return np.where(hi, e_hi, e_lo), np.where(hi, d1_hi, d1_lo), np.where(hi, d2_hi, d2_lo)


def lda_fxc(n):
    """f_xc(n) = d^2(n eps_xc)/dn^2 (Ha bohr^3): Slater exchange plus Perdew-Zunger correlation."""
    n = np.asarray(n, dtype=np.float64)
    fx = -(1.0 / 3.0) * (3.0 / PI) ** (1.0 / 3.0) * n ** (-2.0 / 3.0)
    rs = (3.0 / (4.0 * PI * n)) ** (1.0 / 3.0)
    _, d1, d2 = _pz_derivatives(rs)
    # d/dn = -(rs/(3n)) d/drs:  d^2(n eps)/dn^2 = -(rs/(3n)) [(2/3) eps' - (rs/3) eps'']
    fc = -(rs / (3.0 * n)) * ((2.0 / 3.0) * d1 - (rs / 3.0) * d2)
    return fx + fc


def fxc_matrix(spec, s) -> np.ndarray:
    """F_GG' = |G| f_xc(G, G') |G'|/(4 pi) on the q = 0 sphere (definition above)."""
    dens = np.maximum(realspace_density(spec, s), N_FLOOR)
    f = lda_fxc(dens)
    n1, n2, n3 = spec.fft
    fg = np.fft.fftn(f) / (n1 * n2 * n3)                          # (1/N_r) sum_r f(r) exp(-iG.r)
    g0 = geo.sphere(spec, (0, 0, 0))
    d = g0[:, None, :] - g0[None, :, :]
    fgg = fg[d[..., 0] % n1, d[..., 1] % n2, d[..., 2] % n3]
    p = geo.cart(spec, (0, 0, 0), g0)
    gl = np.sqrt(np.sum(p * p, axis=1))
    return gl[:, None] * fgg * gl[None, :] / (4.0 * PI)


def fxc_pair_kernels(spec, s):
    """The ALDA kernel in the e-h basis, for the coupled-problem check: (Kf, Bf) with
    Kf_SS' = 1/(Omega Nk) sum_GG' conj(rho_S(G)) f_xc(G, G') rho_S'(G') and
    Bf_SS' = 1/(Omega Nk) sum_GG' conj(rho_S(G)) f_xc(G, G') conj(rho_S'(-G')), G, G' != 0."""
    rho = pair.exchange_rho(spec, s.gk, s.coef)
    dens = np.maximum(realspace_density(spec, s), N_FLOOR)
    f = lda_fxc(dens)
    n1, n2, n3 = spec.fft
    fg = np.fft.fftn(f) / (n1 * n2 * n3)
    g0 = geo.sphere(spec, (0, 0, 0))
    d = g0[:, None, :] - g0[None, :, :]
    fgg = fg[d[..., 0] % n1, d[..., 1] % n2, d[..., 2] % n3]
    fgg[0, :] = 0.0
    fgg[:, 0] = 0.0
    mi = coupling.minus_g_index(spec)
    nrm = ok.norm_factor(spec)
    Kf = nrm * np.conj(rho) @ fgg @ rho.T
    Bf = nrm * np.conj(rho) @ fgg @ np.conj(rho[:, mi]).T
    return Kf, Bf
