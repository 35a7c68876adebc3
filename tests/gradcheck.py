"""Finite-difference helpers shared by the GPU gradient tests (no GPU code here)."""
import numpy as np


def w_directions(s, step=4e-2):
    """Two perturbations of W that keep it Hermitian and reciprocal: D1 = W and
    D2 = W_GG'(q) f(|q+G|) f(|q+G'|) with f(p) = cos(1.3 p) + 1/2 (a function of |q+G| only,
    and reciprocity pairs q+G with -(q+G)).  Returns (name, D, h) with the difference step h
    scaled so that no entry of W moves by more than step times itself."""
    from oracle import geometry as geo
    from synth.systems import recip_lattice
    spec = s.spec
    B = recip_lattice(spec)
    kr = geo.mesh_offsets(spec)
    nk = np.asarray(spec.nk)
    f = np.zeros(s.W.shape[:2])
    for iq in range(spec.nkpt):
        gq = s.gq[iq]
        p = (gq + kr[iq] / nk) @ B
        f[iq, :len(gq)] = np.cos(1.3 * np.linalg.norm(p, axis=1)) + 0.5
    W0 = s.W.astype(np.complex128)
    ff = f[:, :, None] * f[:, None, :]
    return W0, [("W", W0, step), ("W f f", W0 * ff, step / float(np.abs(ff).max()))]


def richardson_fd(loss_at, h):
    """Central differences at h and 2h combined to cancel the h^2 term."""
    d1 = (loss_at(h) - loss_at(-h)) / (2 * h)
    d2 = (loss_at(2 * h) - loss_at(-2 * h)) / (4 * h)
    return (4 * d1 - d2) / 3
