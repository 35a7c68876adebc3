"""Oracle: statically screened interaction from the independent-particle response (RPA).

Test infrastructure only (see package docstring).

The screened interaction that step A4 consumes, computed here from the system's own
states instead of the model eps^-1 (Sec. II A-B, Eqs. chi0_GG, epsilon_-1; Sec. III A):

- Adler-Wiser response at w = 0 with the resonant and anti-resonant terms of a
  time-reversal pair of transitions (each 1/(e_v - e_c)) and spin 2:
      chi0_GG'(q) = 4/(Omega Nk) sum_k sum_{v,c} rho(G) conj(rho(G')) / (e_vk - e_c,k+q),
  rho = rho_vc^{k,k+q}(G) = <v k| exp(-i(q+G).r) |c k+q> (Eq. pair_density), k+q unfolded:
  with k' = k+q folded onto the mesh and k+q = k' + G0, rho(G) is the plane-wave
  correlation of (k, v) and (k', c) taken at G + G0.  Bare band energies (no scissor), with
  the dipole's gap floor.  The band sum runs over the system's Nv + Nc bands.
- Symmetrised dielectric matrix eps_GG' = delta_GG' - v^1/2(q+G) chi0_GG' v^1/2(q+G'),
  v^1/2(p) = sqrt(4 pi)/|p| (bulk Coulomb), and W_GG'(q) = v^1/2 eps^-1_GG' v^1/2, the form
  in which the model W is also built.
- q = 0: the G = 0 row and column are the optical limit along qhat: v^1/2(q) rho_S(q + 0)
  -> sqrt(4 pi) conj(P_S) with the k.p dipole P_S of step A6, so that the extended pair
  vector a_S = (sqrt(4 pi) conj(P_S), v^1/2(G) rho_S(G) for G != 0) gives
  eps = 1 - sum_S w_S a_S a_S^H.  The head of W is the spherical mini-zone average
  [eps^-1]_00 12 pi/q_c^2, q_c = (6 pi^2/(Omega Nk))^(1/3), and the wings of W are zero (the
  reading used for the model W).
- Bulk (3D Coulomb) systems only.

Pinned by tests/test_oracle_screening.py: the (k, k+q) pair densities against brute-force
sums over the Born-von Karman supercell (fixes the G0 direction), chi0 Hermitian and negative
semidefinite, eps^-1 against the Woodbury form of the inverse, the head of eps at q = 0
against the Kramers-Kronig static limit of the independent-particle eps_2 of step A8 (fixes
the factor 4/(Omega Nk) against the spectrum's prefactor), and the wings at q = 0 against
the limit q -> 0 along qhat of the same matrix built from finite-q pair densities of true
eigenstates of a model crystal Hamiltonian (for which rho_vc^{k,k+q}(0)/|q| -> conj(P_S),
Eq. density_matrix; the synthetic random states of the workloads are not eigenstates).
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from . import pair

PI = 3.141592653589793


def _gap(spec, e_c, e_v, gap_floor):
    return max(e_c - e_v, gap_floor)


def chi0_pair(spec, s, iq):
    """Pair densities and weights of chi0(q): rho[S][G] (S = (k, v, c)), w[S] = 4/(Omega Nk)/(e_v - e_c')."""
    kr = geo.mesh_offsets(spec)
    nk = np.asarray(spec.nk, dtype=np.int64)
    gq = geo.sphere(spec, tuple(kr[iq]))
    nvc = spec.nv * spec.nc
    rho = np.zeros((spec.dim, len(gq)), dtype=np.complex128)
    w = np.zeros(spec.dim)
    pref = 4.0 / (geo.cell_volume(spec) * spec.nkpt)
    floor = 0.1 / 27.211386245988
    vb = list(range(spec.nv))
    cb = list(range(spec.nv, spec.nb))
    for ik in range(spec.nkpt):
        tot = kr[ik] + kr[iq]
        k2v = np.mod(tot, nk)
        g0 = (tot - k2v) // nk                      # k + q = k' + G0
        ik2 = geo.mesh_index(spec, k2v)
        r = pair.rho_corr(spec, ik, ik2, vb, cb, gq + g0[None, :], s.gk, s.coef)
        rho[ik * nvc:(ik + 1) * nvc] = r.reshape(nvc, -1)
        for iv in range(spec.nv):
            for ic in range(spec.nc):
                de = _gap(spec, s.energies[ik2, spec.nv + ic], s.energies[ik, iv], floor)
                w[geo.pair_index(spec, ik, iv, ic)] = -pref / de
    return gq, rho, w


def sqrt_coulomb(spec, iq):
    """v^1/2(q+G) on the q sphere (0 where q+G = 0)."""
    kr = geo.mesh_offsets(spec)
    gq = geo.sphere(spec, tuple(kr[iq]))
    p = geo.cart(spec, kr[iq], gq)
    n = np.sqrt(np.sum(p * p, axis=1))
    out = np.zeros(len(gq))
    out[n > 0] = np.sqrt(4.0 * PI) / n[n > 0]
    return out


def chi0(spec, s, iq):
    """chi0_GG'(q) (q = 0: the G = 0 row and column are left zero; see epsilon)."""
    _, rho, w = chi0_pair(spec, s, iq)
    return (rho.T * w[None, :]) @ np.conj(rho)


def epsilon(spec, s, iq, P=None):
    """Symmetrised eps_GG'(q); at q = 0 the head and wings from the k.p dipole P (step A6)."""
    _, rho, w = chi0_pair(spec, s, iq)
    vs = sqrt_coulomb(spec, iq)
    a = rho * vs[None, :]                            # v^1/2(q+G) rho_S(G)
    if iq == 0:
        if P is None:
            P = pair.dipole(spec, s.gk, s.coef, s.energies)
        a[:, 0] = np.sqrt(4.0 * PI) * np.conj(P)
    return np.eye(a.shape[1]) - (a.T * w[None, :]) @ np.conj(a)


def screened_w(spec, s, iq, P=None):
    """W_GG'(q) = v^1/2 eps^-1 v^1/2, head at q = 0 by the mini-zone average, wings zero."""
    eps = epsilon(spec, s, iq, P)
    einv = np.linalg.inv(eps)
    vs = sqrt_coulomb(spec, iq)
    W = vs[:, None] * einv * vs[None, :]
    if iq == 0:
        qc = (6.0 * PI * PI / (geo.cell_volume(spec) * spec.nkpt)) ** (1.0 / 3.0)
        W[0, :] = 0.0
        W[:, 0] = 0.0
        W[0, 0] = einv[0, 0] * 12.0 * PI / (qc * qc)
    return W
