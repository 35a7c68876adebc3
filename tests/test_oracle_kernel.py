"""Pins for the oracle's K^x, K^d and Hamiltonian assembly (steps A3-A5)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from synth import SystemSpec

PI = math.pi


def test_exchange_hermitian_psd(cfg1, cfg1_oracle):
    kx = ok.exchange_kernel(cfg1.spec, cfg1_oracle["rho_x"])
    assert np.abs(kx - kx.conj().T).max() < 1e-15
    assert np.linalg.eigvalsh(kx).min() > -1e-14


def test_exchange_single_pair_closed_form():
    """Nk = 1, one v and one c plane wave G_a apart: K^x = 4 pi / (Omega |G_a|^2)."""
    spec = SystemSpec("one", "fcc", 10.0, 0.0, (1, 1, 1), 1, 1, 4.0, (24, 24, 24), "3d")
    g = geo.sphere(spec, (0, 0, 0))
    coef = np.zeros((1, 2, len(g)), complex)
    ia = 5
    coef[0, 0, 0] = 1.0                       # c_v = delta_{G,0}
    coef[0, 1, ia] = 1.0                      # c_c = delta_{G,G_a}
    rx = op.exchange_rho(spec, [g], coef)
    kx = ok.exchange_kernel(spec, rx)
    ga = geo.cart(spec, (0, 0, 0), g[ia:ia + 1])[0]
    assert kx.shape == (1, 1)
    assert abs(kx[0, 0] - 4.0 * PI / (250.0 * ga @ ga)) < 1e-15


def test_full_build_is_hermitian_and_equals_mirrored_assembly(cfg1, cfg1_oracle):
    """Every block built independently: Hermitian only through the reciprocity of W."""
    spec = cfg1.spec
    blocks = [(0, 0), (0, 5), (5, 0), (7, 40), (40, 7), (63, 1), (1, 63), (22, 22)]
    kd = ok.direct_kernel_full(spec, cfg1.gk, cfg1.coef, cfg1.W, blocks=blocks)
    nvc = 9
    H = cfg1_oracle["H"]
    for i, j in [(0, 5), (7, 40), (63, 1)]:
        bij = kd[i * nvc:(i + 1) * nvc, j * nvc:(j + 1) * nvc]
        bji = kd[j * nvc:(j + 1) * nvc, i * nvc:(i + 1) * nvc]
        assert np.abs(bij - bji.conj().T).max() < 1e-15 * max(1.0, np.abs(bij).max()) + 1e-17
        assert np.abs(bij + H[i * nvc:(i + 1) * nvc, j * nvc:(j + 1) * nvc]
                      - 2.0 * ok.exchange_kernel(spec, cfg1_oracle["rho_x"])[i * nvc:(i + 1) * nvc, j * nvc:(j + 1) * nvc]).max() < 1e-15
    for i in (0, 22):
        b = kd[i * nvc:(i + 1) * nvc, i * nvc:(i + 1) * nvc]
        assert np.abs(b - b.conj().T).max() < 1e-15


def test_kernel_off_hamiltonian_is_diagonal(cfg1):
    spec = cfg1.spec
    rx = np.zeros((spec.dim, 113), complex)
    H = ok.hamiltonian_from_factors(spec, cfg1.energies, spec.delta, rx, [], cfg1.W)
    de = ok.transition_energies(spec, cfg1.energies, spec.delta)
    assert np.array_equal(H, np.diag(de).astype(complex))
    assert de[geo.pair_index(spec, 2, 1, 2)] == cfg1.energies[2, 3 + 2] + spec.delta - cfg1.energies[2, 1]


# ---------------------------------------------------------------------------
# Wannier-Mott limit: a thin 2D sheet with parabolic bands and a screened,
# slab-truncated Coulomb W must bind one exciton at E_g - 2 mu / eps^2.
# ---------------------------------------------------------------------------

A_LAT, C_LAT, EPS, EG = 1.0, 0.01, 4.0, 1.0          # m_e = m_h = 1 -> mu = 1/2


def _sheet(n):
    return SystemSpec(f"wm{n}", "hex", A_LAT, C_LAT, (n, n, 1), 1, 1, 80.0, (8, 8, 4), "slab")


def _min_image(spec):
    """Cartesian minimum-image k and the reciprocal vector removed, per k of the mesh."""
    b = geo.reciprocal_basis(spec)
    kr = geo.mesh_offsets(spec)
    red = kr[:, :2] / spec.nk[0]
    best, shift = None, None
    for m1 in (-1, 0, 1):
        for m2 in (-1, 0, 1):
            c = (red - np.array([m1, m2])) @ b[:2, :2]
            if best is None:
                best, shift = c.copy(), np.tile([m1, m2], (len(c), 1))
            else:
                sel = np.sum(c * c, 1) < np.sum(best * best, 1)
                best[sel], shift[sel] = c[sel], [m1, m2]
    return best, shift


def _w_sheet(spec, p):
    """Diagonal model W(p) = v_2D(p)/eps, v_2D = 4 pi/p^2 (1 - exp(-|p| zc)) for in-plane p."""
    zc = 0.5 * spec.c
    q = np.linalg.norm(p, axis=-1)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(q > 0, 4.0 * PI / (q * q) * (1.0 - np.exp(-q * zc)) / EPS, np.nan)


def _head(spec):
    nk = spec.nkpt
    area = spec.a * spec.a * math.sqrt(3.0) / 2.0
    qc = math.sqrt(4.0 * PI / (area * nk))
    x, w = np.polynomial.legendre.leggauss(64)
    q = 0.5 * qc * (x + 1.0)
    f = 2.0 * PI * q * 4.0 * PI * (1.0 - np.exp(-q * 0.5 * spec.c)) / (q * q)
    return 0.5 * qc * np.sum(w * f) / (PI * qc * qc) / EPS


def _analytic_h(n):
    """H_kk' = E(k) delta - W(k - k')/(Omega Nk), k minimum image (textbook Wannier model)."""
    spec = _sheet(n)
    k, _ = _min_image(spec)
    e = EG + np.sum(k * k, 1) / (2.0 * 0.5)
    d = k[:, None, :] - k[None, :, :]
    w = _w_sheet(spec, d)
    w[np.isnan(w)] = _head(spec)
    return np.diag(e) - w / (geo.cell_volume(spec) * spec.nkpt)


def test_oracle_direct_kernel_equals_wannier_model():
    """Oracle pipeline on plane-wave states (c_vk = delta_{G,-G(k)}, c_ck = delta_{G,b1-G(k)})."""
    n = 6
    spec = _sheet(n)
    kr = geo.mesh_offsets(spec)
    kmin, shift = _min_image(spec)
    gk = [geo.sphere(spec, tuple(o)) for o in kr]
    npw = max(len(g) for g in gk)
    coef = np.zeros((spec.nkpt, 2, npw), complex)
    for ik in range(spec.nkpt):
        lut = {tuple(g): t for t, g in enumerate(gk[ik])}
        coef[ik, 0, lut[(-shift[ik, 0], -shift[ik, 1], 0)]] = 1.0
        coef[ik, 1, lut[(1 - shift[ik, 0], -shift[ik, 1], 0)]] = 1.0
    ngmax = max(len(geo.sphere(spec, tuple(o))) for o in kr)
    W = np.zeros((spec.nkpt, ngmax, ngmax), complex)
    for iq in range(spec.nkpt):
        g = geo.sphere(spec, tuple(kr[iq]))
        p = geo.cart(spec, kr[iq], g)
        w = _w_sheet(spec, p[:, :2])
        if iq == 0:
            w[0] = _head(spec)
        W[iq, :len(g), :len(g)] = np.diag(w)
    e = np.zeros((spec.nkpt, 2))
    e[:, 0] = -np.sum(kmin * kmin, 1) / 2.0
    e[:, 1] = EG + np.sum(kmin * kmin, 1) / 2.0
    kd = ok.direct_kernel_full(spec, gk, coef, W)
    H = np.diag(ok.transition_energies(spec, e, 0.0)).astype(complex) - kd
    assert np.abs(H - _analytic_h(n)).max() < 1e-12


def test_wannier_model_binds_2d_hydrogen():
    """Richardson (1/n) extrapolation of the lowest eigenvalue -> E_g - 2 mu/eps^2 within 2%."""
    ns = np.array([48, 64, 80, 96], dtype=float)
    eb = []
    for n in ns.astype(int):
        e0 = sla.eigsh(_analytic_h(n), k=1, which="SA", tol=1e-12)[0][0]
        eb.append(EG - e0)
    c = np.polyfit(1.0 / ns, np.array(eb), 1)
    exact = 2.0 * 0.5 / EPS ** 2
    assert abs(c[1] - exact) / exact < 0.02
