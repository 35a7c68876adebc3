"""Pins for the oracle's spectrum (steps A7, A8)."""
import math

import numpy as np

from oracle import kernel as ok
from oracle import spectrum as osp
from oracle import geometry as geo

PI = math.pi


def test_haydock_full_dimension_equals_dense_eig(cfg1, cfg1_oracle):
    spec = cfg1.spec
    H, P = cfg1_oracle["H"], cfg1_oracle["P"]
    e1 = osp.eps2_dense(spec, H, P, cfg1.omega, spec.eta)
    e2, a, b, done = osp.eps2_haydock(spec, H, P, cfg1.omega, spec.eta, spec.dim)
    assert done == spec.dim
    assert np.abs(e1 - e2).max() / np.abs(e1).max() < 1e-10


def test_kernel_off_equals_adler_wiser_resonant_term(cfg1, cfg1_oracle):
    """K = 0: eps_2 = -(4 pi/q^2) Im chi0_00 (Eq. chi0_GG, resonant v->c terms, spin 2, 1/Nk)."""
    spec = cfg1.spec
    P = cfg1_oracle["P"]
    de = ok.transition_energies(spec, cfg1.energies, spec.delta)
    H = np.diag(de).astype(complex)
    w = cfg1.omega
    q = 1e-3                                             # |n_S(0)| = |q| |P_S|
    n0 = np.abs(P) * q
    omega_cell = geo.cell_volume(spec)
    chi0 = np.zeros(len(w), complex)
    for s in range(spec.dim):
        f_occ, f_emp = 1.0, 0.0
        chi0 += (2.0 / (omega_cell * spec.nkpt)) * (f_occ - f_emp) * n0[s] ** 2 / (w - de[s] + 1j * spec.eta)
    ref = -(4.0 * PI / q ** 2) * chi0.imag
    for got in (osp.eps2_dense(spec, H, P, w, spec.eta), osp.eps2_haydock(spec, H, P, w, spec.eta, spec.dim)[0]):
        assert np.abs(got - ref).max() / ref.max() < 1e-10


def test_moments_and_finite_window_sum_rule(cfg1, cfg1_oracle):
    spec = cfg1.spec
    H, P = cfg1_oracle["H"], cfg1_oracle["P"]
    e, a = np.linalg.eigh(H)
    wts = np.abs(np.conj(P) @ a) ** 2
    assert abs(wts.sum() - np.vdot(P, P).real) < 1e-12 * wts.sum()
    assert abs((e * wts).sum() - np.vdot(P, H @ P).real) < 1e-12 * abs((e * wts).sum())
    ah, bh, _, _ = osp.haydock(H, P, 5)
    assert abs(ah[0] * np.vdot(P, P).real - (e * wts).sum()) < 1e-12 * abs((e * wts).sum())
    # integral over a finite window of the Lorentzian-broadened spectrum, closed form
    w = np.linspace(0.0, 0.4, 40001)
    eps2 = osp.eps2_dense(spec, H, P, w, spec.eta)
    integral = np.sum(0.5 * (eps2[1:] + eps2[:-1]) * np.diff(w))
    closed = osp.prefactor(spec) * np.sum(wts * (np.arctan((w[-1] - e) / spec.eta) - np.arctan((w[0] - e) / spec.eta)))
    assert abs(integral - closed) / closed < 1e-7
    assert abs(osp.prefactor(spec) - 8.0 * PI / (250.0 * 64)) < 1e-18


def test_scissor_shift_is_rigid(cfg1, cfg1_oracle):
    spec = cfg1.spec
    H, P = cfg1_oracle["H"], cfg1_oracle["P"]
    s = 0.013
    w = cfg1.omega
    e_a = osp.eps2_haydock(spec, H + s * np.eye(spec.dim), P, w, spec.eta, 100)[0]
    e_b = osp.eps2_haydock(spec, H, P, w - s, spec.eta, 100)[0]
    assert np.abs(e_a - e_b).max() / np.abs(e_b).max() < 1e-11


def test_breakdown_on_invariant_subspace_is_exact(cfg1):
    spec = cfg1.spec
    rng = np.random.default_rng(5)
    m = rng.standard_normal((12, 12)) + 1j * rng.standard_normal((12, 12))
    H = np.zeros((40, 40), complex)
    H[:12, :12] = 0.01 * (m + m.conj().T) + np.diag(np.linspace(0.1, 0.3, 12))
    H[12:, 12:] = np.diag(np.linspace(0.05, 0.35, 28))
    P = np.zeros(40, complex)
    P[:12] = rng.standard_normal(12)
    w = np.linspace(0, 0.4, 300)
    got, a, b, done = osp.eps2_haydock(spec, H, P, w, 0.004, 30)
    assert done == 12
    ref = osp.eps2_dense(spec, H, P, w, 0.004)
    assert np.abs(got - ref).max() / ref.max() < 1e-10


def test_ritz_pairs_pinned(cfg1, cfg1_oracle):
    """Ritz values/weights of the Haydock tridiagonal: dense eigenvalues of T, sum w = 1,
    sum w theta = a_0, sum w theta^2 = a_0^2 + b_1^2, the pole expansion equals the continued
    fraction, and at full Krylov dimension they are H's eigenvalues with weights |P^H A|^2/|P|^2."""
    H, P = cfg1_oracle["H"], cfg1_oracle["P"]
    a, b, done, _ = osp.haydock(H, P, 60)
    th, w = osp.ritz(a, b)
    T = np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1)
    assert np.abs(np.sort(np.linalg.eigvalsh(T)) - th).max() < 1e-12
    assert abs(w.sum() - 1.0) < 1e-12
    assert abs(w @ th - a[0]) < 1e-12
    assert abs(w @ th ** 2 - (a[0] ** 2 + b[1] ** 2)) < 1e-12
    z = np.linspace(0.0, 0.5, 41) + 1j * 0.01
    g = osp.continued_fraction(a, b, z)
    assert np.abs((w[None, :] / (z[:, None] - th[None, :])).sum(1) - g).max() < 1e-9 * np.abs(g).max()
    # full Krylov dimension: the Ritz pairs are H's eigenpairs with nonzero weight
    a, b, done, _ = osp.haydock(H, P, H.shape[0])
    th, w = osp.ritz(a, b)
    e, v = np.linalg.eigh(H)
    wt = np.abs(np.conj(P) @ v) ** 2 / np.vdot(P, P).real
    keep = w > 1e-8
    for t, x in zip(th[keep], w[keep]):
        i = np.argmin(np.abs(e - t))
        assert abs(e[i] - t) < 1e-9 and abs(wt[i] - x) < 1e-7 * max(1.0, x)
