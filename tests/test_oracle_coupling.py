"""Pins of oracle/coupling.py (the BSE with e-h / h-e coupling, Appendix A)."""
import numpy as np
import pytest

from oracle import coupling as cp
from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp
from synth import generate


@pytest.fixture(scope="module")
def tiny(tiny_spec):
    s = generate(tiny_spec)
    spec = s.spec
    rho_x = op.exchange_rho(spec, s.gk, s.coef)
    A = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rho_x, ok.direct_factors(spec, s.gk, s.coef), s.W)
    B = cp.coupling_full(spec, s.gk, s.coef, s.W)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    return s, rho_x, A, B, P


def test_coupling_pair_densities_match_realspace_sums(tiny):
    """rho_vc'^{kk'} (v at k, c' at k') and rho_cv'^{kk'} against (1/N_r) sum_r conj(u) u exp(-iG.r)."""
    s = tiny[0]
    spec = s.spec
    kr = geo.mesh_offsets(spec)
    for ik, ik2 in ((0, 0), (0, 5), (3, 6), (7, 1)):
        iq, rvc, rcv = cp.coupling_rho_block(spec, ik, ik2, s.gk, s.coef)
        _, iqv, g0 = geo.fold(spec, kr[ik], kr[ik2])
        gt = geo.sphere(spec, tuple(iqv)) - g0[None, :]
        for iv in range(spec.nv):
            for ic in range(spec.nc):
                ref = op.rho_realspace(spec, ik, ik2, iv, spec.nv + ic, gt, s.gk, s.coef)
                assert np.abs(rvc[iv, ic] - ref).max() < 1e-12
                ref = op.rho_realspace(spec, ik, ik2, spec.nv + ic, iv, gt, s.gk, s.coef)
                assert np.abs(rcv[ic, iv] - ref).max() < 1e-12


def test_exchange_coupling_uses_the_h_e_pair_density(tiny):
    """Bx_SS' = 1/(Omega Nk) sum_{G != 0} conj(rho_vc^{kk}(G)) vbar(G) rho_c'v'^{k'k'}(G), the h-e density
    summed in real space (so the conj(rho(-G)) form and the -G index are checked)."""
    s, rho_x = tiny[0], tiny[1]
    spec = s.spec
    bx = cp.exchange_coupling(spec, rho_x)
    g0 = geo.sphere(spec, (0, 0, 0))
    v = ok.coulomb_bar(spec)
    for S2 in (0, 7, 13, 30):
        k2, iv2, ic2 = S2 // (spec.nv * spec.nc), (S2 // spec.nc) % spec.nv, S2 % spec.nc
        rhe = op.rho_realspace(spec, k2, k2, spec.nv + ic2, iv2, g0, s.gk, s.coef)   # rho_c'v'(G)
        ref = ok.norm_factor(spec) * (np.conj(rho_x) * v[None, :]) @ rhe
        assert np.abs(bx[:, S2] - ref).max() < 1e-12 * np.abs(bx).max()


def test_coupling_symmetric_from_independent_blocks(tiny):
    s, rho_x, _, B, _ = tiny
    spec = s.spec
    bx = cp.exchange_coupling(spec, rho_x)
    bd = cp.coupling_direct_full(spec, s.gk, s.coef, s.W)
    for m in (bx, bd, B):
        assert np.abs(m - m.T).max() < 1e-12 * np.abs(m).max()
    assert np.abs(bd).max() > 1e-3 * np.abs(bx).max()        # both parts present


def test_assembly_from_upper_blocks_equals_independent_build(tiny):
    s, rho_x, _, B, _ = tiny
    spec = s.spec
    b2 = cp.coupling_from_factors(spec, rho_x, cp.coupling_factors(spec, s.gk, s.coef), s.W)
    assert np.abs(b2 - B).max() < 1e-12 * np.abs(B).max()


def test_h2_spectrum_in_plus_minus_pairs_and_positive_metric(tiny):
    _, _, A, B, _ = tiny
    dim = A.shape[0]
    e = np.linalg.eigvals(cp.h2(A, B))
    assert np.abs(e.imag).max() < 1e-9 * np.abs(e).max()
    er = np.sort(e.real)
    assert np.abs(er + er[::-1]).max() < 1e-9 * np.abs(er).max()
    M = cp.f_sign(dim)[:, None] * cp.h2(A, B)
    assert np.abs(M - M.conj().T).max() < 1e-13 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0


def test_one_pair_closed_form(tiny_spec):
    """dim 1: A = a, B = b.  (z - H2)^{-1} by hand gives Q(z) = 2 (a|p|^2 + Re(conj(b) p^2)) / (z^2 - a^2 + |b|^2)."""
    a, b, p = 0.31, 0.07 - 0.05j, 0.6 + 0.8j
    A = np.array([[a]], dtype=np.complex128)
    Bm = np.array([[b]], dtype=np.complex128)
    P = np.array([p])
    w = np.linspace(0.0, 0.6, 61)
    eta = 0.01
    z = w + 1j * eta
    q = 2.0 * (a * abs(p) ** 2 + (np.conj(b) * p * p).real) / (z * z - a * a + abs(b) ** 2)
    ref = -osp.prefactor(tiny_spec) * q.imag
    assert np.abs(cp.eps2_direct(tiny_spec, A, Bm, P, w, eta) - ref).max() < 1e-12 * np.abs(ref).max()
    e2, al, bl, done, s2 = cp.eps2_lanczos(tiny_spec, A, Bm, P, w, eta, 2)
    assert done == 2 and abs(al).max() < 1e-14
    assert abs(bl[1] - np.sqrt(a * a - abs(b) ** 2)) < 1e-14
    assert np.abs(e2 - ref).max() < 1e-12 * np.abs(ref).max()


def test_no_coupling_gives_resonant_minus_antiresonant(tiny):
    s, _, A, _, P = tiny
    spec = s.spec
    w = np.linspace(-0.1, 0.5, 121)
    eta = spec.eta
    e, v = np.linalg.eigh(A)
    wts = np.abs(np.conj(P) @ v) ** 2
    lor = lambda x: eta / (x * x + eta * eta)   # noqa: E731
    ref = osp.prefactor(spec) * (lor(w[:, None] - e[None, :]) - lor(w[:, None] + e[None, :])) @ wts
    got = cp.eps2_direct(spec, A, np.zeros_like(A), P, w, eta)
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_lanczos_at_full_krylov_dimension_equals_direct_solve(tiny):
    s, _, A, B, P = tiny
    spec = s.spec
    w = np.linspace(0.0, 0.5, 101)
    ref = cp.eps2_direct(spec, A, B, P, w, spec.eta)
    got, a, b, done, _ = cp.eps2_lanczos(spec, A, B, P, w, spec.eta, 2 * spec.dim)
    assert np.abs(got - ref).max() < 1e-9 * np.abs(ref).max()
    assert np.abs(a).max() < 1e-10 * b[1:].max()                # +- symmetric measure: zero diagonal
    # the coupling moves the spectrum: the TDA value differs by far more than the tolerance
    tda = osp.eps2_dense(spec, A, P, w, spec.eta)
    assert np.abs(tda - ref).max() > 1e-3 * np.abs(ref).max()


def test_spectrum_odd_in_frequency(tiny):
    s, _, A, B, P = tiny
    spec = s.spec
    w = np.linspace(0.01, 0.4, 40)
    ep = cp.eps2_direct(spec, A, B, P, w, spec.eta)
    em = cp.eps2_direct(spec, A, B, P, -w, spec.eta)
    assert np.abs(ep + em).max() < 1e-12 * np.abs(ep).max()


def test_half_vector_recursion_equals_full_m_lanczos(tiny):
    """The recursion the CUDA path runs: only e-h halves x_j of the Lanczos vectors, q_j = (x_j, +-conj x_j)
    with alternating parity, t = A x + s B conj(x), |q|_M^2 = 2 Re(x^H t), reorthogonalisation against every
    stored vector with <q_i, w>_M = 2 Re d (same parity) or 2i Im d (other parity), d = p_i^H y, and no
    diagonal coefficient.  In FP64 it reproduces the oracle's full 2 dim M-Lanczos coefficients."""
    s, _, A, B, P = tiny
    n = 40
    a_ref, b_ref, done, s2 = cp.m_lanczos(A, B, P, n)
    assert done == n
    X, Pp = [], []                       # stored x_i and p_i = t_i / b_i (e-h halves)
    b = np.zeros(n)
    w = P.astype(np.complex128).copy()   # e-h half of s = F Pt = (P, conj P)
    q_prev = None
    for j in range(n):
        sg = 1.0 if j % 2 == 0 else -1.0
        t = A @ w + sg * (B @ np.conj(w))
        beta2 = 2.0 * np.vdot(w, t).real
        b[j] = np.sqrt(beta2)
        q, p = w / b[j], t / b[j]
        X.append(q)
        Pp.append(p)
        if j + 1 == n:
            break
        w = p - (b[j] * q_prev if q_prev is not None else 0.0)
        for _ in range(2):
            c = []
            for i in range(j + 1):
                d = np.vdot(Pp[i], w)
                c.append(2.0 * d.real if (i - (j + 1)) % 2 == 0 else 2j * d.imag)
            w = w - sum(ci * xi for ci, xi in zip(c, X))
        q_prev = q
    assert abs(b[0] ** 2 - s2) < 1e-12 * s2
    assert np.abs(b[1:] - b_ref[1:]).max() < 1e-11 * b_ref.max()
    assert np.abs(a_ref).max() < 1e-10 * b_ref.max()
