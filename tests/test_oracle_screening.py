"""Pins of oracle/screening.py (RPA screening from the independent-particle response)."""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import pair as op
from oracle import screening as scr
from oracle import spectrum as osp
from synth import generate


@pytest.fixture(scope="module")
def tiny(tiny_spec):
    return generate(tiny_spec)


def _psi_supercell(spec, ik, band, gk, coef):
    """psi_nk on the Born-von Karman supercell grid (unnormalised), by explicit plane-wave sums."""
    n = np.asarray(spec.fft) * np.asarray(spec.nk)
    x = np.stack(np.meshgrid(*[np.arange(m) / float(f) for m, f in zip(n, spec.fft)], indexing="ij"), -1).reshape(-1, 3)
    kr = geo.mesh_offsets(spec)[ik] / np.asarray(spec.nk, dtype=np.float64)
    g = np.asarray(gk[ik], dtype=np.float64)
    c = coef[ik, band, : len(g)]
    return np.exp(2j * np.pi * (x @ (g + kr[None, :]).T)) @ c, x


def test_k_kq_pair_densities_match_supercell_matrix_elements(tiny):
    """rho(G) = <v k| exp(-i(q+G).r) |c k+q> summed over the whole Born-von Karman supercell."""
    spec = tiny.spec
    kr = geo.mesh_offsets(spec)
    for iq in (1, 3, 6):
        gq, rho, _ = scr.chi0_pair(spec, tiny, iq)
        qred = kr[iq] / np.asarray(spec.nk, dtype=np.float64)
        for ik in (0, 5, 7):
            k2 = geo.mesh_index(spec, np.mod(kr[ik] + kr[iq], np.asarray(spec.nk)))
            for iv in range(spec.nv):
                pv, x = _psi_supercell(spec, ik, iv, tiny.gk, tiny.coef)
                for ic in range(spec.nc):
                    pc, _ = _psi_supercell(spec, k2, spec.nv + ic, tiny.gk, tiny.coef)
                    ph = np.exp(-2j * np.pi * (x @ (gq + qred[None, :]).T))       # exp(-i(q+G).r)
                    ref = (np.conj(pv) * pc) @ ph / len(x)
                    got = rho[geo.pair_index(spec, ik, iv, ic)]
                    assert np.abs(got - ref).max() < 1e-12


def test_chi0_hermitian_negative_semidefinite(tiny):
    spec = tiny.spec
    for iq in (0, 2, 7):
        c = scr.chi0(spec, tiny, iq)
        assert np.abs(c - c.conj().T).max() < 1e-14 * np.abs(c).max()
        ev = np.linalg.eigvalsh(c)
        assert ev.max() < 1e-12 * np.abs(ev).max()
        assert ev.min() < 0


def test_inverse_dielectric_matches_woodbury(tiny):
    """eps = I + B B^H (B = a^T diag(sqrt(-w))): eps^-1 = I - B (I + B^H B)^-1 B^H; eigenvalues of eps >= 1."""
    spec = tiny.spec
    P = op.dipole(spec, tiny.gk, tiny.coef, tiny.energies)
    for iq in (0, 4):
        _, rho, w = scr.chi0_pair(spec, tiny, iq)
        a = rho * scr.sqrt_coulomb(spec, iq)[None, :]
        if iq == 0:
            a[:, 0] = np.sqrt(4.0 * np.pi) * np.conj(P)
        B = a.T * np.sqrt(-w)[None, :]
        wood = np.eye(B.shape[0]) - B @ np.linalg.solve(np.eye(B.shape[1]) + B.conj().T @ B, B.conj().T)
        eps = scr.epsilon(spec, tiny, iq, P)
        assert np.linalg.eigvalsh(eps).min() > 1.0 - 1e-12
        assert np.abs(np.linalg.inv(eps) - wood).max() < 1e-10
        W = scr.screened_w(spec, tiny, iq, P)
        assert np.abs(W - W.conj().T).max() < 1e-12 * np.abs(W).max()


def test_head_matches_kramers_kronig_of_independent_particle_spectrum(tiny):
    """eps_00(q -> 0) - 1 = (2/pi) int_0^inf eps_2(w)/w dw for the independent-particle eps_2 of step A8
    (resonant and anti-resonant Lorentzians; eta small), computed by numerical quadrature."""
    spec = tiny.spec
    P = op.dipole(spec, tiny.gk, tiny.coef, tiny.energies)
    e = tiny.energies
    de = np.array([max(e[ik, spec.nv + ic] - e[ik, iv], 0.1 / 27.211386245988)
                   for ik in range(spec.nkpt) for iv in range(spec.nv) for ic in range(spec.nc)])
    eta = 2e-4
    w = np.concatenate([np.linspace(0.0, 2.0, 400001)[1:], np.linspace(2.0, 400.0, 400001)[1:]])
    eps2 = osp.eps2_independent(spec, de, P, w, eta) - osp.eps2_independent(spec, de, P, -w, eta)
    f = eps2 / w
    integral = np.sum(0.5 * (f[1:] + f[:-1]) * np.diff(w)) + 0.5 * f[0] * w[0]
    kk = 2.0 / np.pi * integral
    head = scr.epsilon(spec, tiny, 0, P)[0, 0].real - 1.0
    assert abs(kk - head) < 2e-3 * head
