"""Oracle: e-h exchange K^x, screened direct K^d and the TDA Hamiltonian (steps A3-A5).

Test infrastructure only (see package docstring).

Readings of the paper (Sec. II C, Eqs. kernel, V_eh, W_SS; Appendix A):
- Singlet Tamm-Dancoff Hamiltonian in the vertical (q = 0) e-h basis
  S = (k, v, c):  H = diag(e_ck + Delta - e_vk) + 2 K^x - K^d, the factor 2 on
  the exchange being the spin factor of Eq. kernel (V - W/2 per spin channel).
- K^x_SS' = 1/(Omega Nk) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) rho_v'c'^{k'k'}(G):
  the short-range exchange Vbar of Eq. V_eh (G = 0 dropped) in the optical
  limit q -> 0, with vbar(G) = 4 pi/|G|^2 (3D) or the slab-truncated 2D form.
- K^d_SS' = 1/(Omega Nk) sum_{G,G'} conj(rho_vv'^{kk'}(G)) W_GG'(k'-k) rho_cc'^{kk'}(G')
  (Eq. W_SS with m = c at k, n = v).  W carries its 4 pi once (Sec. III A form).
- 1/Nk: Bloch states normalised over the Born-von Karman supercell of Nk cells.

``hamiltonian_full`` builds every (k, k') block independently from the
coefficients, with no mirroring, so that Hermiticity of the result is a real
test of the reciprocity of W (Eq. for W under time reversal, Sec. III A, with
T = identity).  ``hamiltonian_from_factors`` is the assembly definition of step
A5 (upper blocks k <= k' from given pair densities, lower blocks by H_k'k =
H_kk'^H, diagonal blocks (B + B^H)/2); the tests pin it to ``hamiltonian_full``.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from . import pair

PI = 3.141592653589793


def coulomb_bar(spec) -> np.ndarray:
    """vbar(G) on the q = 0 sphere (G = 0 excluded -> 0)."""
    g0 = geo.sphere(spec, (0, 0, 0))
    p = geo.cart(spec, (0, 0, 0), g0)
    p2 = np.sum(p * p, axis=1)
    v = np.zeros(len(g0))
    nz = p2 > 0
    if spec.coulomb == "3d":
        v[nz] = 4.0 * PI / p2[nz]
    else:
        zc = 0.5 * spec.c
        ppar = np.sqrt(p[:, 0] ** 2 + p[:, 1] ** 2)
        v[nz] = 4.0 * PI / p2[nz] * (1.0 - np.exp(-ppar[nz] * zc) * np.cos(p[nz, 2] * zc))
    return v


def norm_factor(spec) -> float:
    return 1.0 / (geo.cell_volume(spec) * spec.nkpt)


def exchange_kernel(spec, rho_x) -> np.ndarray:
    """K^x = 1/(Omega Nk) rho_x^H diag(vbar) rho_x  with rho_x[S][G]."""
    v = coulomb_bar(spec)
    return norm_factor(spec) * (np.conj(rho_x) * v[None, :]) @ rho_x.T


def direct_block(spec, rv, rc, w) -> np.ndarray:
    """K^d block [(v,c),(v',c')] from rho~_vv' [v][v'][p], rho~_cc' [c][c'][p], W(q) [p][p']."""
    m = np.einsum("abp,pq,cdq->abcd", np.conj(rv), w, rc, optimize=True)      # [v][v'][c][c']
    nv, nc = rv.shape[0], rc.shape[0]
    return norm_factor(spec) * m.transpose(0, 2, 1, 3).reshape(nv * nc, nv * nc)


def w_of_q(spec, W, iq) -> np.ndarray:
    ng = len(geo.sphere(spec, tuple(geo.mesh_offsets(spec)[iq])))
    return np.asarray(W[iq, :ng, :ng], dtype=np.complex128)


def direct_kernel_full(spec, gk, coef, W, blocks=None) -> np.ndarray:
    """K^d from every (k, k') block computed independently (no mirroring)."""
    nvc = spec.nv * spec.nc
    kd = np.zeros((spec.dim, spec.dim), dtype=np.complex128)
    if blocks is None:
        blocks = [(i, j) for i in range(spec.nkpt) for j in range(spec.nkpt)]
    for ik, ik2 in blocks:
        iq, rv, rc = pair.direct_rho_block(spec, ik, ik2, gk, coef)
        kd[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] = direct_block(spec, rv, rc, w_of_q(spec, W, iq))
    return kd


def transition_energies(spec, energies, delta) -> np.ndarray:
    """e_ck + Delta - e_vk on the pair index S = (k, v, c)."""
    ev = energies[:, : spec.nv]
    ec = energies[:, spec.nv:]
    return (ec[:, None, :] + delta - ev[:, :, None]).reshape(-1)


def hamiltonian_full(spec, gk, coef, energies, W, delta) -> np.ndarray:
    rho_x = pair.exchange_rho(spec, gk, coef)
    kx = exchange_kernel(spec, rho_x)
    kd = direct_kernel_full(spec, gk, coef, W)
    return np.diag(transition_energies(spec, energies, delta)).astype(np.complex128) + 2.0 * kx - kd


def direct_factors(spec, gk, coef) -> list:
    """[(ik, ik', iq, rv, rc)] for the upper blocks ik <= ik' (row-major)."""
    out = []
    for ik, ik2 in geo.upper_blocks(spec):
        iq, rv, rc = pair.direct_rho_block(spec, ik, ik2, gk, coef)
        out.append((ik, ik2, iq, rv, rc))
    return out


def hamiltonian_from_factors(spec, energies, delta, rho_x, factors, W) -> np.ndarray:
    """Step A5 from given pair densities: upper blocks, mirrored lower blocks."""
    nvc = spec.nv * spec.nc
    h = 2.0 * exchange_kernel(spec, rho_x)
    h = h + np.diag(transition_energies(spec, energies, delta))
    for ik, ik2, iq, rv, rc in factors:
        blk = h[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] - direct_block(spec, rv, rc, w_of_q(spec, W, iq))
        if ik == ik2:
            blk = 0.5 * (blk + blk.conj().T)
        h[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] = blk
        if ik != ik2:
            h[ik2 * nvc:(ik2 + 1) * nvc, ik * nvc:(ik + 1) * nvc] = blk.conj().T
    return h
