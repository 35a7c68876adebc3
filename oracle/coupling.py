"""Oracle: the Bethe-Salpeter problem beyond the Tamm-Dancoff approximation (Appendix A).

Test infrastructure only (see package docstring).

Appendix A keeps both e-h transitions S = (v -> c) and h-e transitions
S-bar = (c -> v) in the two-particle basis.  With the occupation factor
f_S = +1 (e-h), -1 (h-e) and transition energy e_c - e_v (+ scissor) the
effective Hamiltonian (Eq. Dyson_eh_rearrange and the definition below it)
takes the block form, in the basis (e-h, h-e),

    H2 = [[ A,        B      ],
          [-conj(B), -conj(A)]]

- A is the Tamm-Dancoff Hamiltonian of ``kernel.py`` (e-h with e-h).
- B_SS' = 2 Bx_SS' - Bd_SS' couples the e-h pair S = (k, v, c) with the h-e
  pair S'-bar = (k', c' -> v').  The pair density of S'-bar is
  rho_c'v'^{k'k'}(G) = conj(rho_v'c'^{k'k'}(-G)), and Eqs. V_eh and W_SS with
  the band labels of S'-bar give

    Bx_SS' = 1/(Omega Nk) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) conj(rho_v'c'^{k'k'}(-G))
    Bd_SS' = 1/(Omega Nk) sum_{G,G'} conj(rho_vc'^{kk'}(G)) W_GG'(k'-k) rho_cv'^{kk'}(G')

  on the same G-sphere and fold (p = q_unf + G) as the direct term of A.
- The h-e rows are the complex conjugates of the e-h rows.  That holds for a
  kernel that is real in real space: vbar is, and W is exactly when it obeys
  the reciprocity W_{-G,-G'}(-q) = conj(W_GG'(q)) that the synthetic W is built
  with.  The same reciprocity makes B symmetric (B^T = B), which is tested,
  with every block built independently.

Spectrum.  Eq. Dyson_eh_rearrange puts f_S' = F = diag(1, -1) on the right of
the resolvent; with Eq. epsilon_chi_bar and the optical matrix element of the
h-e pair, n_{S-bar}(0) = -conj(n_S(0)) to first order in q,

    eps_2(w) = -C Im[ Pt^H (z - H2)^{-1} F Pt ],   Pt = (P, -conj(P)),  z = w + i eta,

C = 8 pi/(Omega Nk) as in the Tamm-Dancoff form (``spectrum.py``), to which it
reduces for B = 0 up to the anti-resonant Lorentzians at -E.

Evaluations:
- ``eps2_direct``: the definition, one linear solve per frequency (small cases).
- ``m_lanczos`` + ``eps2_lanczos``: M = F H2 = [[A, B], [conj(B), conj(A)]] is
  Hermitian and, for a stable system, positive definite; H2 is self-adjoint in
  the inner product <x, y>_M = x^H M y.  Lanczos in that inner product from
  s = F Pt, with classical Gram-Schmidt applied twice against the whole basis
  (projections <q_i, w>_M = (F H2 q_i)^H w), gives a real tridiagonal T and
  g(z) = e_0^T (z - T)^{-1} e_0.  Because Pt^H F Pt = 0 and F^2 = 1,
  <s, (z - H2)^{-1} s>_M = Pt^H H2 (z - H2)^{-1} F Pt = z Q(z) with
  Q(z) = Pt^H (z - H2)^{-1} F Pt, so eps_2 = -C |s|_M^2 Im[g(z)/z].
  a_j = <q_j, H2 q_j>_M is computed as (H2 q_j)^H F (H2 q_j) (one product per
  step).  Breakdown: beta_{j+1} <= 1e-10 |H2 q_j|_M; a negative squared norm
  beyond rounding means M is not positive definite (ValueError).

Pinned by tests/test_oracle_coupling.py: B symmetric from independent blocks,
assembly from upper blocks equal to the independent build, coupling pair
densities against the brute-force real-space sum, eigenvalues of H2 in +-
pairs, B = 0 reduces to the resonant minus anti-resonant closed form, Lanczos
at full Krylov dimension equal to the direct solve, a_j = 0 (the +-symmetric
spectral measure of s), eps_2 odd in w.
"""
from __future__ import annotations

import numpy as np

from . import geometry as geo
from . import kernel as ok
from . import pair
from . import spectrum as osp

BREAKDOWN_REL = 1e-10


def minus_g_index(spec) -> np.ndarray:
    """Index of -G on the q = 0 sphere (the sphere is symmetric under inversion)."""
    g0 = geo.sphere(spec, (0, 0, 0))
    pos = {tuple(int(x) for x in g): i for i, g in enumerate(g0)}
    return np.array([pos[tuple(int(-x) for x in g)] for g in g0], dtype=np.int64)


def exchange_coupling(spec, rho_x) -> np.ndarray:
    """Bx = 1/(Omega Nk) conj(rho_x) diag(vbar) conj(rho_x[:, -G])^T  with rho_x[S][G]."""
    v = ok.coulomb_bar(spec)
    mi = minus_g_index(spec)
    return ok.norm_factor(spec) * (np.conj(rho_x) * v[None, :]) @ np.conj(rho_x[:, mi]).T


def coupling_rho_block(spec, ik, ik2, gk, coef):
    """rho~_vc'^{kk'}[p] and rho~_cv'^{kk'}[p] on the sphere of q = fold(k'-k), G = g_p - G0.

    Returns (iq, rvc [Nv][Nc][NG] (v at k, c' at k'), rcv [Nc][Nv][NG] (c at k, v' at k')).
    """
    kr = geo.mesh_offsets(spec)
    iq, iqv, g0 = geo.fold(spec, kr[ik], kr[ik2])
    gp = geo.sphere(spec, tuple(iqv))
    gt = gp - g0[None, :]
    vb = list(range(spec.nv))
    cb = list(range(spec.nv, spec.nb))
    rvc = pair.rho_corr(spec, ik, ik2, vb, cb, gt, gk, coef)
    rcv = pair.rho_corr(spec, ik, ik2, cb, vb, gt, gk, coef)
    return iq, rvc, rcv


def coupling_direct_block(spec, rvc, rcv, w) -> np.ndarray:
    """Bd block [(v,c),(v',c')] = 1/(Omega Nk) sum conj(rvc[v][c'][p]) w[p][p'] rcv[c][v'][p']."""
    m = np.einsum("aip,pq,bjq->aibj", np.conj(rvc), w, rcv, optimize=True)     # [v][c'][c][v']
    nv, nc = rvc.shape[0], rvc.shape[1]
    return ok.norm_factor(spec) * m.transpose(0, 2, 3, 1).reshape(nv * nc, nv * nc)


def coupling_direct_full(spec, gk, coef, W, blocks=None) -> np.ndarray:
    """Bd from every (k, k') block computed independently (no mirroring)."""
    nvc = spec.nv * spec.nc
    bd = np.zeros((spec.dim, spec.dim), dtype=np.complex128)
    if blocks is None:
        blocks = [(i, j) for i in range(spec.nkpt) for j in range(spec.nkpt)]
    for ik, ik2 in blocks:
        iq, rvc, rcv = coupling_rho_block(spec, ik, ik2, gk, coef)
        bd[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] = coupling_direct_block(spec, rvc, rcv,
                                                                                      ok.w_of_q(spec, W, iq))
    return bd


def coupling_full(spec, gk, coef, W) -> np.ndarray:
    """B = 2 Bx - Bd with every block independent."""
    rho_x = pair.exchange_rho(spec, gk, coef)
    return 2.0 * exchange_coupling(spec, rho_x) - coupling_direct_full(spec, gk, coef, W)


def coupling_factors(spec, gk, coef) -> list:
    """[(ik, ik', iq, rvc, rcv)] for the upper blocks ik <= ik' (row-major)."""
    out = []
    for ik, ik2 in geo.upper_blocks(spec):
        iq, rvc, rcv = coupling_rho_block(spec, ik, ik2, gk, coef)
        out.append((ik, ik2, iq, rvc, rcv))
    return out


def coupling_from_factors(spec, rho_x, factors, W) -> np.ndarray:
    """Assembly from upper blocks: B_k'k = B_kk'^T, diagonal blocks (B + B^T)/2."""
    nvc = spec.nv * spec.nc
    b = 2.0 * exchange_coupling(spec, rho_x)
    for ik, ik2, iq, rvc, rcv in factors:
        blk = (b[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc]
               - coupling_direct_block(spec, rvc, rcv, ok.w_of_q(spec, W, iq)))
        if ik == ik2:
            blk = 0.5 * (blk + blk.T)
        b[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] = blk
        if ik != ik2:
            b[ik2 * nvc:(ik2 + 1) * nvc, ik * nvc:(ik + 1) * nvc] = blk.T
    return b


def h2(A, B) -> np.ndarray:
    return np.block([[A, B], [-np.conj(B), -np.conj(A)]])


def p_tilde(P) -> np.ndarray:
    return np.concatenate([P, -np.conj(P)])


def f_sign(dim) -> np.ndarray:
    return np.concatenate([np.ones(dim), -np.ones(dim)])


def eps2_direct(spec, A, B, P, omega, eta) -> np.ndarray:
    """-C Im[Pt^H (z - H2)^{-1} F Pt] by one dense solve per frequency."""
    dim = len(P)
    H = h2(A, B)
    pt = p_tilde(P)
    rhs = f_sign(dim) * pt
    out = np.zeros(len(omega))
    eye = np.eye(2 * dim)
    for i, w in enumerate(omega):
        x = np.linalg.solve((w + 1j * eta) * eye - H, rhs)
        out[i] = -osp.prefactor(spec) * np.vdot(pt, x).imag
    return out


def m_lanczos(A, B, P, nsteps):
    """Lanczos of H2 in the M = F H2 inner product from s = F Pt (CGS2 each step).

    Returns (a [n], b [n], steps_done, s_norm2); b[0] = 0, b[j] couples q_{j-1} and q_j.
    """
    dim = len(P)
    F = f_sign(dim)

    def apply(x):                                 # H2 x from the blocks; conj(M) y = conj(M conj(y))
        top, bot = x[:dim], x[dim:]
        return np.concatenate([A @ top + B @ bot, -np.conj(B @ np.conj(top) + A @ np.conj(bot))])

    nsteps = min(nsteps, 2 * dim)
    s = F * p_tilde(P)
    u = apply(s)
    s_norm2 = np.vdot(s, F * u).real
    if not s_norm2 > 0.0:
        raise ValueError("|s|_M^2 <= 0: M = F H2 is not positive definite (or P = 0)")
    beta = np.sqrt(s_norm2)
    Q = np.zeros((nsteps, 2 * dim), dtype=np.complex128)      # q_j
    MQ = np.zeros((nsteps, 2 * dim), dtype=np.complex128)     # M q_j = F H2 q_j
    a = np.zeros(nsteps)
    b = np.zeros(nsteps)
    q, p = s / beta, u / beta
    done = nsteps
    for j in range(nsteps):
        Q[j], MQ[j] = q, F * p
        a[j] = np.vdot(p, F * p).real
        if j + 1 == nsteps:
            break
        w = p - a[j] * q - (b[j] * Q[j - 1] if j > 0 else 0.0)
        for _ in range(2):
            h = np.conj(MQ[: j + 1] @ np.conj(w))       # (M q_i)^H w for every i <= j
            w = w - Q[: j + 1].T @ h
        u = apply(w)
        beta2 = np.vdot(w, F * u).real
        scale2 = a[j] ** 2 + b[j] ** 2 + abs(beta2)            # |H2 q_j|_M^2 in exact arithmetic
        if beta2 <= (BREAKDOWN_REL ** 2) * scale2:
            if beta2 < -1e-8 * scale2:
                raise ValueError("negative M-norm: M = F H2 is not positive definite")
            done = j + 1
            break
        b[j + 1] = np.sqrt(beta2)
        q, p = w / b[j + 1], u / b[j + 1]
    return a[:done], b[:done], done, s_norm2


def eps2_lanczos(spec, A, B, P, omega, eta, nsteps):
    """eps_2 = -C |s|_M^2 Im[g(z)/z] from ``m_lanczos``; returns (eps2, a, b, done, s_norm2)."""
    a, b, done, s2 = m_lanczos(A, B, P, nsteps)
    z = omega + 1j * eta
    g = osp.continued_fraction(a, b, z)
    return -osp.prefactor(spec) * s2 * (g / z).imag, a, b, done, s2
