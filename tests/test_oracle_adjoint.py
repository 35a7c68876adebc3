"""Pins for the oracle gradient (step A9): central finite differences of the oracle forward."""
import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import kernel as ok
from oracle import pair as op
from oracle import geometry as geo
from synth import generate


@pytest.fixture(scope="module")
def tiny(tiny_spec):
    spec = tiny_spec.replace(eta=0.01)
    s = generate(spec)
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    w = np.linspace(0.0, 0.6, 200)
    H0 = ok.hamiltonian_from_factors(spec, s.energies, 0.9 * spec.delta, rx, fac, s.W)
    from oracle.spectrum import eps2_dense
    target = eps2_dense(spec, H0, P, w, spec.eta)
    weight = np.full(len(w), 1.0 / len(w))
    return spec, s, rx, fac, P, w, target, weight


def _loss(tiny, delta=None, rx=None, fac=None, W=None):
    spec, s, rx0, fac0, P, w, target, weight = tiny
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta if delta is None else delta,
                                    rx0 if rx is None else rx, fac0 if fac is None else fac,
                                    s.W if W is None else W)
    return oa.spectral_loss(spec, H, P, w, spec.eta, target, weight)


def _grads(tiny):
    spec, s, rx, fac, P, w, target, weight = tiny
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    _, g = oa.spectral_loss(spec, H, P, w, spec.eta, target, weight)
    return oa.gradients(spec, s.energies, spec.delta, rx, fac, s.W, P, w, spec.eta, g)


def test_delta_gradient_fd(tiny):
    spec = tiny[0]
    d_delta = _grads(tiny)[0]
    h = 1e-6
    fd = (_loss(tiny, delta=spec.delta + h)[0] - _loss(tiny, delta=spec.delta - h)[0]) / (2 * h)
    assert abs(d_delta - fd) < 1e-5 * abs(fd)


def test_rho_gradients_fd(tiny):
    spec, s, rx, fac = tiny[:4]
    _, drx, dfac, _, _ = _grads(tiny)
    h = 1e-6
    for (i, j) in [(0, 3), (17, 10), (31, 0)]:
        for unit in (1.0, 1j):
            rp, rm = rx.copy(), rx.copy()
            rp[i, j] += h * unit
            rm[i, j] -= h * unit
            fd = (_loss(tiny, rx=rp)[0] - _loss(tiny, rx=rm)[0]) / (2 * h)
            an = drx[i, j].real if unit == 1.0 else drx[i, j].imag
            assert abs(an - fd) < 1e-4 * abs(fd) + 1e-8
    for (b, which, idx) in [(0, 3, (0, 1, 2)), (5, 4, (1, 1, 0)), (11, 3, (1, 0, 4))]:
        for unit in (1.0, 1j):
            fp = [list(f) for f in fac]
            fm = [list(f) for f in fac]
            fp[b][which] = fp[b][which].copy()
            fm[b][which] = fm[b][which].copy()
            fp[b][which][idx] += h * unit
            fm[b][which][idx] -= h * unit
            fd = (_loss(tiny, fac=[tuple(f) for f in fp])[0] - _loss(tiny, fac=[tuple(f) for f in fm])[0]) / (2 * h)
            g = dfac[b][which - 3][idx]
            an = g.real if unit == 1.0 else g.imag
            assert abs(an - fd) < 1e-4 * abs(fd) + 1e-8


def test_w_independent_entry_gradient_fd(tiny):
    spec, s = tiny[0], tiny[1]
    dW = _grads(tiny)[3]
    kr = geo.mesh_offsets(spec)
    n = np.asarray(spec.nk)
    h = 1e-6
    for iq, i, j in [(0, 1, 4), (1, 0, 2), (3, 2, 2), (6, 1, 3)]:
        iqbv = np.mod(-kr[iq], n)
        iqb = geo.mesh_index(spec, iqbv)
        if iqb < iq:
            continue
        g0p = (-kr[iq] - iqbv) // n
        gq = geo.sphere(spec, tuple(kr[iq]))
        lut = {tuple(g): t for t, g in enumerate(geo.sphere(spec, tuple(iqbv)))}
        pi_i, pi_j = lut[tuple(g0p - gq[i])], lut[tuple(g0p - gq[j])]

        def perturbed(d):
            W = s.W.copy()
            theta = W[iq, i, j] + d
            imgs_t = {(iq, i, j), (iqb, pi_j, pi_i)}
            imgs_c = {(iq, j, i), (iqb, pi_i, pi_j)} - imgs_t
            for e in imgs_t:
                W[e] = theta
            for e in imgs_c:
                W[e] = np.conj(theta)
            return W
        fd = (_loss(tiny, W=perturbed(h))[0] - _loss(tiny, W=perturbed(-h))[0]) / (2 * h)
        an = oa.independent_w_gradient(spec, dW, iq, i, j).real
        assert abs(an - fd) < 1e-4 * abs(fd) + 1e-8
