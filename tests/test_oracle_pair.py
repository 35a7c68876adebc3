"""Pins for the oracle's pair densities and dipole (steps A2, A6)."""
import numpy as np

from oracle import geometry as geo
from oracle import pair
from synth import generate


def test_orthonormality_gives_delta_at_g0(cfg1):
    """rho_nn'^{kk}(G=0) = <psi_n|psi_n'> = delta_nn' (Eq. pair_density at q = G = 0)."""
    spec = cfg1.spec
    for ik in (0, 17, 63):
        r = pair.rho_corr(spec, ik, ik, list(range(6)), list(range(6)), np.zeros((1, 3), int), cfg1.gk, cfg1.coef)
        assert np.abs(r[:, :, 0] - np.eye(6)).max() < 1e-13


def test_correlation_equals_bruteforce_realspace(tiny_spec):
    """Eq. (1) by G-space correlation equals the explicit real-space sum on an alias-free 8^3 grid."""
    s = generate(tiny_spec)
    spec = tiny_spec
    for ik, ik2 in [(0, 0), (0, 5), (3, 6), (7, 2)]:
        kr = geo.mesh_offsets(spec)
        _, iqv, g0 = geo.fold(spec, kr[ik], kr[ik2])
        gt = geo.sphere(spec, tuple(iqv)) - g0[None, :]
        a = pair.rho_corr(spec, ik, ik2, [0, 1, 2, 3], [0, 1, 2, 3], gt, s.gk, s.coef)
        for n, m in [(0, 0), (1, 3), (3, 2)]:
            b = pair.rho_realspace(spec, ik, ik2, n, m, gt, s.gk, s.coef)
            assert np.abs(a[n, m] - b).max() < 1e-13


def test_pair_density_reciprocity(cfg1):
    """rho_mn^{k'k}(G) = conj(rho_nm^{kk'}(-G))."""
    spec = cfg1.spec
    g = geo.sphere(spec, (0, 0, 0))[:40]
    a = pair.rho_corr(spec, 3, 40, [0, 1, 4], [2, 5], g, cfg1.gk, cfg1.coef)
    b = pair.rho_corr(spec, 40, 3, [2, 5], [0, 1, 4], -g, cfg1.gk, cfg1.coef)
    assert np.abs(a - np.conj(b).transpose(1, 0, 2)).max() < 1e-14


def test_dipole_single_plane_wave_closed_form(tiny_spec):
    """One plane wave per band: P = conj(qhat.(k+G) delta_{G_v,G_c}) / (e_c - e_v) -> known value."""
    spec = tiny_spec.replace(nv=1, nc=1)
    kr = geo.mesh_offsets(spec)
    gk = [geo.sphere(spec, tuple(o)) for o in kr]
    npw = max(len(g) for g in gk)
    coef = np.zeros((spec.nkpt, 2, npw), complex)
    coef[:, 0, 0] = 1.0
    coef[:, 1, 0] = 1j                       # same G: <v|grad|c> nonzero
    e = np.tile([[-0.1, 0.3]], (spec.nkpt, 1))
    p = pair.dipole(spec, gk, coef, e)
    for ik in range(spec.nkpt):
        kg = geo.cart(spec, kr[ik], gk[ik][:1])[0, 0]
        assert abs(p[ik] - np.conj(1j * kg) / 0.4) < 1e-14
