"""Oracle: pair densities (charge density matrix), step A2 and the dipole of step A6.

Test infrastructure only (see package docstring).

Eq. pair_density defines n_{nk,n'k+q}(G) = <psi_nk| exp(-i(q+G).r) |psi_n'k+q>.
With psi_nk(r) = Omega^{-1/2} sum_G c_nk(G) exp(i(k+G).r) and k' = k+q taken
unfolded, the integral collapses to the plane-wave correlation

    rho_nm^{kk'}(G) = sum_{G1 in S(k)} conj(c_nk(G1)) c_mk'(G1+G)      (1)

(zero where G1+G is outside S(k')).  ``rho_corr`` evaluates (1) directly - no
FFT - so the CUDA path's FFT route is checked against a different formula.
``rho_realspace`` is the brute-force real-space sum (1/N_r) sum_r conj(u) u
exp(-iG.r) with u built by explicit exponential sums; it pins (1) on tiny grids.

The k.p optical limit (Eq. density_matrix) gives, for q -> 0 along qhat,
n_{vk,ck+q}(0)/|q| = qhat . sum_G conj(c_vk(G)) (k+G) c_ck(G) / (e_ck - e_vk).
The spectrum (Eq. epsilon_chi_bar) contracts n_S(0) on the left and n*_S'(0)
on the right, so the vector entering P^H R P is P_S = conj(n_S(0))/|q|.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo


def _box_coefs(spec, ik, gk, coef):
    """Place the coefficients of k on a dense G box (zero outside the sphere)."""
    g = gk[ik]
    n = len(g)
    lo = g.min(axis=0)
    hi = g.max(axis=0)
    return lo, hi, g, coef[ik, :, :n]


def rho_corr(spec, ik, ik2, bands_n, bands_m, gtargets, gk, coef) -> np.ndarray:
    """Eq. (1) for n in bands_n (at k), m in bands_m (at k'), G in gtargets -> [n][m][G]."""
    g1 = np.asarray(gk[ik], dtype=np.int64)
    c1 = coef[ik, :, : len(g1)][bands_n]
    g2 = np.asarray(gk[ik2], dtype=np.int64)
    c2 = coef[ik2, :, : len(g2)][bands_m]
    gt = np.asarray(gtargets, dtype=np.int64)
    lo = np.minimum(g2.min(axis=0), (g1.min(axis=0) + gt.min(axis=0))) - 1
    hi = np.maximum(g2.max(axis=0), (g1.max(axis=0) + gt.max(axis=0))) + 1
    shape = tuple(int(x) for x in (hi - lo + 1))
    nbox = shape[0] * shape[1] * shape[2]
    strides = np.array([shape[1] * shape[2], shape[2], 1], dtype=np.int64)
    box = np.zeros((nbox, len(bands_m)), dtype=np.complex128)     # c_mk' on the box, bands innermost
    box[(g2 - lo) @ strides] = c2.T
    # c_mk'(G1 + G) for every (G1, G): the box position of G1 + G - lo is the sum of the positions of
    # G1 - lo and of G (row-major strides of the box)
    pos = ((g1 - lo) @ strides)[:, None] + (gt @ strides)[None, :]   # [G1][G]
    shifted = box[pos].reshape(len(g1), len(gt) * len(bands_m))       # [G1][(G, m)]
    # sum over G1 of conj(c_nk(G1)) c_mk'(G1 + G), as one matrix product over the G1 axis
    r = (np.conj(c1) @ shifted).reshape(len(bands_n), len(gt), len(bands_m))     # [n][G][m]
    return np.ascontiguousarray(r.transpose(0, 2, 1))


def wavefunction_realspace(spec, ik, band, gk, coef) -> np.ndarray:
    """u~_nk(r_j) = sum_G c_nk(G) exp(2 pi i G.j/N) by explicit sums (tiny grids only)."""
    n1, n2, n3 = spec.fft
    g = np.asarray(gk[ik], dtype=np.int64)
    c = coef[ik, band, : len(g)]
    j = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    phase = 2.0 * np.pi * (np.outer(j[:, 0], g[:, 0]) / n1 + np.outer(j[:, 1], g[:, 1]) / n2
                           + np.outer(j[:, 2], g[:, 2]) / n3)
    return (np.exp(1j * phase) @ c).reshape(n1, n2, n3)


def rho_realspace(spec, ik, ik2, n, m, gtargets, gk, coef) -> np.ndarray:
    """(1/N_r) sum_r conj(u_nk) u_mk' exp(-iG.r) by explicit sums (tiny grids only)."""
    n1, n2, n3 = spec.fft
    prod = (np.conj(wavefunction_realspace(spec, ik, n, gk, coef))
            * wavefunction_realspace(spec, ik2, m, gk, coef)).reshape(-1)
    j = np.stack(np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3), indexing="ij"), -1).reshape(-1, 3)
    gt = np.asarray(gtargets, dtype=np.int64)
    phase = 2.0 * np.pi * (np.outer(gt[:, 0], j[:, 0]) / n1 + np.outer(gt[:, 1], j[:, 1]) / n2
                           + np.outer(gt[:, 2], j[:, 2]) / n3)
    return (np.exp(-1j * phase) @ prod) / (n1 * n2 * n3)


def exchange_rho(spec, gk, coef) -> np.ndarray:
    """rho_x[S][G] = rho_{vc}^{kk}(G), S = (k,v,c), G on the q = 0 sphere."""
    g0 = geo.sphere(spec, (0, 0, 0))
    out = np.zeros((spec.dim, len(g0)), dtype=np.complex128)
    vb = list(range(spec.nv))
    cb = list(range(spec.nv, spec.nb))
    for ik in range(spec.nkpt):
        r = rho_corr(spec, ik, ik, vb, cb, g0, gk, coef)           # [v][c][G]
        out[ik * spec.nv * spec.nc:(ik + 1) * spec.nv * spec.nc] = r.reshape(spec.nv * spec.nc, -1)
    return out


def direct_rho_block(spec, ik, ik2, gk, coef):
    """rho~_vv'^{kk'}[p] and rho~_cc'^{kk'}[p] on the sphere of q = fold(k'-k).

    Index p runs over the W sphere of the folded q; the pair density is taken at
    G = g_p - G0 so that q_unf + G = q + g_p (W(k'-k)_{GG'} = W(q)_{G+G0,G'+G0}).
    Returns (iq, rv [Nv][Nv][NG], rc [Nc][Nc][NG]).
    """
    kr = geo.mesh_offsets(spec)
    iq, iqv, g0 = geo.fold(spec, kr[ik], kr[ik2])
    gp = geo.sphere(spec, tuple(iqv))
    gt = gp - g0[None, :]
    vb = list(range(spec.nv))
    cb = list(range(spec.nv, spec.nb))
    rv = rho_corr(spec, ik, ik2, vb, vb, gt, gk, coef)
    rc = rho_corr(spec, ik, ik2, cb, cb, gt, gk, coef)
    return iq, rv, rc


def dipole(spec, gk, coef, energies, qhat=(1.0, 0.0, 0.0), gap_floor=0.1 / 27.211386245988) -> np.ndarray:
    """P_S = conj(qhat . sum_G conj(c_vk) (k+G) c_ck) / max(e_ck - e_vk, gap_floor)  (Eq. density_matrix).

    Bare band energies (no scissor), so a scissor shift moves the spectrum rigidly.
    """
    kr = geo.mesh_offsets(spec)
    qh = np.asarray(qhat, dtype=np.float64)
    out = np.zeros(spec.dim, dtype=np.complex128)
    for ik in range(spec.nkpt):
        g = gk[ik]
        kg = geo.cart(spec, kr[ik], g) @ qh                               # qhat.(k+G)
        c = coef[ik, :, : len(g)]
        for iv in range(spec.nv):
            for ic in range(spec.nc):
                m = np.sum(np.conj(c[iv]) * kg * c[spec.nv + ic])
                de = max(energies[ik, spec.nv + ic] - energies[ik, iv], gap_floor)
                out[geo.pair_index(spec, ik, iv, ic)] = np.conj(m) / de
    return out
