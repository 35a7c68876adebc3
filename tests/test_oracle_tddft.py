"""Pins of oracle/tddft.py (macroscopic dielectric function from TDDFT with local fields)."""
import numpy as np
import pytest

from oracle import coupling
from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp
from oracle import tddft as td
from synth import SystemSpec, generate


@pytest.fixture(scope="module")
def small():
    spec = SystemSpec("td", "fcc", 10.0, 0.0, (2, 2, 2), 2, 2, 2.0, (12, 12, 12), "3d", nsteps=20, nw=60)
    return generate(spec)


def _omega(spec):
    return np.linspace(0.05, 1.2, 41)


def _bse_eps_m(spec, s, omega, eta, A, B, P):
    """eps_M = 1 - C Pt^H (z - H2)^-1 F Pt of the coupled e-h problem (Appendix A), complex."""
    H = coupling.h2(A, B)
    pt = coupling.p_tilde(P)
    rhs = coupling.f_sign(len(P)) * pt
    out = np.zeros(len(omega), dtype=np.complex128)
    for i, w in enumerate(omega):
        x = np.linalg.solve((w + 1j * eta) * np.eye(2 * len(P)) - H, rhs)
        out[i] = 1.0 - osp.prefactor(spec) * np.vdot(pt, x)
    return out


def test_no_local_fields_is_the_independent_particle_spectrum(small):
    """Im(1 - chi~0_00) = eps_2^IP(w) - eps_2^IP(-w) with the closed form of step A8 (kernel off)."""
    spec = small.spec
    om = _omega(spec)
    eta = 0.01
    chi0 = td.chi0_bar(spec, small, om, eta, spec.delta)
    P = op.dipole(spec, small.gk, small.coef, small.energies)
    de = ok.transition_energies(spec, small.energies, spec.delta)
    ref = osp.eps2_independent(spec, de, P, om, eta) - osp.eps2_independent(spec, de, P, -om, eta)
    got = td.epsilon_macro_nlf(chi0).imag
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # chi~0(w)^H is chi~0 at the conjugate frequency w - i eta
    conj_z = td.chi0_bar(spec, small, om[:3], -eta, spec.delta, P)
    assert np.abs(conj_z - np.conj(np.transpose(chi0[:3], (0, 2, 1)))).max() < 1e-12 * np.abs(chi0).max()


def test_rpa_local_fields_equal_exchange_only_coupled_bse(small):
    """eps_M from the Dyson equation with K = v and the inversion 1/[eps^-1]_00 equals 1 minus the response
    of the coupled e-h problem whose kernel is the exchange alone: A = diag + 2 K^x, B = 2 Bx."""
    spec = small.spec
    om = _omega(spec)
    eta = 0.01
    P = op.dipole(spec, small.gk, small.coef, small.energies)
    chi0 = td.chi0_bar(spec, small, om, eta, spec.delta, P)
    eps = td.epsilon_macro(chi0)
    rx = op.exchange_rho(spec, small.gk, small.coef)
    A = np.diag(ok.transition_energies(spec, small.energies, spec.delta)) + 2.0 * ok.exchange_kernel(spec, rx)
    B = 2.0 * coupling.exchange_coupling(spec, rx)
    ref = _bse_eps_m(spec, small, om, eta, A, B, P)
    assert np.abs(eps - ref).max() < 1e-9 * np.abs(ref).max()
    # local fields matter here (the check is not the trivial one)
    assert np.abs(eps - td.epsilon_macro_nlf(chi0)).max() > 1e-3 * np.abs(ref).max()


def test_alda_local_fields_equal_coupled_bse_with_xc_kernel(small):
    """With K = v + f_xc the same identity holds with 2 (K^x + K^f) and 2 (Bx + B^f) in the e-h basis."""
    spec = small.spec
    om = _omega(spec)
    eta = 0.01
    P = op.dipole(spec, small.gk, small.coef, small.energies)
    chi0 = td.chi0_bar(spec, small, om, eta, spec.delta, P)
    F = td.fxc_matrix(spec, small)
    assert np.abs(F - F.conj().T).max() < 1e-12 * np.abs(F).max()
    assert np.all(F[0] == 0) and np.all(F[:, 0] == 0)
    eps = td.epsilon_macro(chi0, F)
    rx = op.exchange_rho(spec, small.gk, small.coef)
    Kf, Bf = td.fxc_pair_kernels(spec, small)
    A = (np.diag(ok.transition_energies(spec, small.energies, spec.delta))
         + 2.0 * (ok.exchange_kernel(spec, rx) + Kf))
    B = 2.0 * (coupling.exchange_coupling(spec, rx) + Bf)
    ref = _bse_eps_m(spec, small, om, eta, A, B, P)
    assert np.abs(eps - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.abs(eps - td.epsilon_macro(chi0)).max() > 1e-4 * np.abs(ref).max()


def test_density_holds_two_electrons_per_valence_band(small):
    spec = small.spec
    n = td.realspace_density(spec, small)
    assert n.min() >= 0.0
    assert abs(n.sum() * geo.cell_volume(spec) / n.size - 2.0 * spec.nv) < 1e-10


def test_xc_kernel_is_the_second_derivative_of_n_eps_xc():
    n = np.array([1e-4, 3e-3, 0.01, 0.05, 0.2, 1.0, 5.0])        # rs from ~13 to ~0.36: both branches
    h = 1e-4 * n
    fd = ((n + h) * td.lda_eps_xc(n + h) - 2.0 * n * td.lda_eps_xc(n) + (n - h) * td.lda_eps_xc(n - h)) / h ** 2
    assert np.abs(td.lda_fxc(n) - fd).max() < 1e-5 * np.abs(fd).max()
    assert np.all(np.abs(td.lda_fxc(n) - fd) < 1e-4 * np.abs(fd))
    # Slater exchange, closed form -(1/3)(3/pi)^(1/3) n^(-2/3), dominates at high density (rs < 1.7)
    fx = -(1.0 / 3.0) * (3.0 / np.pi) ** (1.0 / 3.0) * n ** (-2.0 / 3.0)
    hi = n >= 0.05
    assert np.all(np.abs(td.lda_fxc(n) - fx)[hi] < 0.1 * np.abs(fx)[hi])


def test_perdew_zunger_branches_meet_at_rs_one():
    e_hi = td.PZ_GAMMA / (1.0 + td.PZ_BETA1 + td.PZ_BETA2)
    e_lo = td.PZ_B + td.PZ_D
    assert abs(e_hi - e_lo) < 1e-3 * abs(e_hi)          # the fit is continuous to 5e-4
    d_hi = -td.PZ_GAMMA * (td.PZ_BETA1 / 2.0 + td.PZ_BETA2) / (1.0 + td.PZ_BETA1 + td.PZ_BETA2) ** 2
    d_lo = td.PZ_A + td.PZ_C + td.PZ_D
    assert abs(d_hi - d_lo) < 1e-3 * abs(d_hi)
    # the correlation energy of the uniform gas is a few tens of mHa per electron around rs ~ 1-5
    rs = np.array([1.0, 2.0, 5.0])
    ec, _, _ = td._pz_derivatives(rs)
    assert np.all(ec < -0.02) and np.all(ec > -0.07)


def test_uniform_density_gives_diagonal_kernel(small):
    """f_xc constant in r -> f_xc(G, G') = f delta_GG' and F = diag(|G|^2 f/(4 pi))."""
    spec = small.spec

    class Flat:
        pass
    flat = Flat()
    flat.gk = [np.zeros((1, 3), dtype=np.int64) for _ in range(spec.nkpt)]
    flat.coef = np.zeros((spec.nkpt, spec.nb, 1), dtype=np.complex128)
    flat.coef[:, :, 0] = 1.0                    # u = 1: a constant density 2 Nv/Omega
    F = td.fxc_matrix(spec, flat)
    n0 = 2.0 * spec.nv / geo.cell_volume(spec)
    g0 = geo.sphere(spec, (0, 0, 0))
    p = geo.cart(spec, (0, 0, 0), g0)
    ref = np.diag(np.sum(p * p, axis=1) * td.lda_fxc(n0) / (4.0 * np.pi))
    assert np.abs(F - ref).max() < 1e-12 * np.abs(ref).max()
