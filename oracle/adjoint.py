"""Oracle: gradient of a spectral loss with respect to Delta, W and the pair densities (step A9).

Test infrastructure only (see package docstring).

The spectrum eps_2(w) = -C Im[P^H R(z) P], R(z) = (z - H)^{-1} (Eq.
epsilon_chi_bar in the TDA, resolvent of Appendix A).  For a loss L(eps_2) with
g(w) = dL/deps_2(w), a perturbation dH gives dL = Re sum_ij conj(G_ij) dH_ij with

    G = -C sum_w g(w) i xt(w) x(w)^H,   x = R(z) P,  xt = R(z)^H P = R(conj z) P,

evaluated here by dense eigendecomposition, R(z) = sum_l A_l A_l^H / (z - E_l)
(Eq. resolvent).  Complex gradients follow dL/dRe + i dL/dIm.

The chain from H to (Delta, rho_x, rho_dir, W) uses PyTorch CPU autograd
through a plain restatement of the assembly of step A5 (``torch_hamiltonian``),
so the hand-derived transposed contractions of the CUDA path are checked
against an independent derivation.  The gradient with respect to W is the one
for each stored entry taken as free; tests compare it after projecting onto the
independent entries (Hermitian and reciprocity images move together).

Pinned by tests/test_oracle_adjoint.py (central finite differences of the
oracle's own forward on a tiny system).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import torch

from . import geometry as geo
from . import kernel as okern
from .spectrum import prefactor


def resolvent_vectors(H, P, omega, eta):
    """x(w) = R(z)P and xt(w) = R(conj z)P for all w, by eigendecomposition -> [nw][dim] each."""
    e, a = scipy.linalg.eigh(H)
    pa = np.conj(a).T @ P                                    # A^H P
    z = omega + 1j * eta
    x = (pa[None, :] / (z[:, None] - e[None, :])) @ a.T
    xt = (pa[None, :] / (np.conj(z)[:, None] - e[None, :])) @ a.T
    return x, xt


def grad_h(spec, H, P, omega, eta, g) -> np.ndarray:
    """G = -C sum_w g(w) i xt(w) x(w)^H (dense)."""
    x, xt = resolvent_vectors(H, P, omega, eta)
    return -prefactor(spec) * 1j * (xt.T * g[None, :]) @ np.conj(x)


def torch_hamiltonian(spec, energies, delta, rho_x, factors, W):
    """Step A5 restated in torch: H = diag(de + Delta) + 2 K^x - K^d (upper blocks, mirrored)."""
    nvc = spec.nv * spec.nc
    nrm = okern.norm_factor(spec)
    v = torch.as_tensor(okern.coulomb_bar(spec), dtype=torch.float64)
    de = torch.as_tensor(okern.transition_energies(spec, energies, 0.0), dtype=torch.float64)
    kx = nrm * (torch.conj(rho_x) * v[None, :]) @ rho_x.T
    h = 2.0 * kx + torch.diag((de + delta).to(torch.complex128))
    blocks = {}
    for n, (ik, ik2, iq, rv, rc) in enumerate(factors):
        ng = rv.shape[-1]
        w = W[iq, :ng, :ng]
        m = torch.einsum("abp,pq,cdq->abcd", torch.conj(rv), w, rc)
        kd = nrm * m.permute(0, 2, 1, 3).reshape(nvc, nvc)
        blk = h[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc] - kd
        if ik == ik2:
            blk = 0.5 * (blk + blk.conj().T)
        blocks[(ik, ik2)] = blk
    rows = []
    nk = spec.nkpt
    for i in range(nk):
        row = []
        for j in range(nk):
            if (i, j) in blocks:
                row.append(blocks[(i, j)])
            elif (j, i) in blocks:
                row.append(blocks[(j, i)].conj().T)
            else:
                row.append(h[i * nvc:(i + 1) * nvc, j * nvc:(j + 1) * nvc])
        rows.append(torch.cat(row, dim=1))
    return torch.cat(rows, dim=0)


def gradients(spec, energies, delta, rho_x, factors, W, P, omega, eta, g):
    """(dL/dDelta, dL/drho_x, [dL/drv, dL/drc per factor], dL/dW) for eps_2 from the dense resolvent."""
    t_delta = torch.tensor(float(delta), dtype=torch.float64, requires_grad=True)
    t_rx = torch.tensor(rho_x, dtype=torch.complex128, requires_grad=True)
    t_W = torch.tensor(np.asarray(W, dtype=np.complex128), requires_grad=True)
    t_f = []
    for ik, ik2, iq, rv, rc in factors:
        t_f.append((ik, ik2, iq, torch.tensor(rv, dtype=torch.complex128, requires_grad=True),
                    torch.tensor(rc, dtype=torch.complex128, requires_grad=True)))
    H = torch_hamiltonian(spec, energies, t_delta, t_rx, t_f, t_W)
    G = torch.as_tensor(grad_h(spec, H.detach().numpy(), P, omega, eta, g))
    surrogate = torch.sum(torch.conj(G) * H).real
    surrogate.backward()
    dfac = [(f[3].grad.resolve_conj().numpy(), f[4].grad.resolve_conj().numpy()) for f in t_f]
    return (float(t_delta.grad), t_rx.grad.resolve_conj().numpy(), dfac, t_W.grad.resolve_conj().numpy(),
            H.detach().resolve_conj().numpy())


def spectral_loss(spec, H, P, omega, eta, target, weight):
    """L = sum_w weight(w) (eps_2(w) - target(w))^2 with the dense spectrum; returns (L, dL/deps_2)."""
    from .spectrum import eps2_dense
    e2 = eps2_dense(spec, H, P, omega, eta)
    r = e2 - target
    return float(np.sum(weight * r * r)), 2.0 * weight * r


def independent_w_gradient(spec, dW, iq, i, j):
    """Gradient with respect to the independent entry W_q[i][j] (q <= qbar, i <= j) from free-entry dW.

    Images that move with W_q[i][j] = theta: (q, i, j) -> theta, (q, j, i) -> conj(theta),
    (qbar, pi(i), pi(j)) -> conj(theta), (qbar, pi(j), pi(i)) -> theta, pi: G -> G0' - G.
    The gradient is sum over theta-images of dW + sum over conj-images of conj(dW) (each image once).
    """
    kr = geo.mesh_offsets(spec)
    n = np.asarray(spec.nk)
    iqv = kr[iq]
    iqbv = np.mod(-iqv, n)
    iqb = geo.mesh_index(spec, iqbv)
    g0p = (-iqv - iqbv) // n
    gq = geo.sphere(spec, tuple(iqv))
    gqb = geo.sphere(spec, tuple(iqbv))
    lut = {tuple(g): t for t, g in enumerate(gqb)}
    pi_i = lut[tuple(g0p - gq[i])]
    pi_j = lut[tuple(g0p - gq[j])]
    theta_imgs = {(iq, i, j), (iqb, pi_j, pi_i)}
    conj_imgs = {(iq, j, i), (iqb, pi_i, pi_j)}
    conj_imgs -= theta_imgs
    tot = sum(dW[e] for e in theta_imgs) + sum(np.conj(dW[e]) for e in conj_imgs)
    if i == j and iq == iqb and pi_i == i:
        return complex(tot.real, 0.0)
    return complex(tot)
