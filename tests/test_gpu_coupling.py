"""The BSE with e-h / h-e coupling (beyond the Tamm-Dancoff approximation) against the oracle.

Coupling pair densities and B within 1e-5 of their max entry (FP32), 1e-4 with BF16x3 products;
the Lanczos coefficients b_j and eps_2 of the coupled spectrum within 1e-5 of the oracle's FP64
recursion on the same A and B, and within 1e-5 of the oracle's independent build end to end.
"""
import numpy as np
import pytest

from oracle import coupling as cp
from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from synth import config_spec, generate

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_1206_3518_gb300 import bse as b
    return b


def _dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _coupled(bse, sysd, nsteps, prec=0, qchunk=None):
    from paper_1206_3518_gb300.pipeline import Coupled, Forward
    spec = sysd.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=nsteps, nw=len(sysd.omega), qchunk=qchunk)
    W = _dev(sysd.W, torch.complex64)
    F.build(_dev(sysd.coef, torch.complex64), _dev(sysd.energies, torch.float64), W, spec.delta, prec)
    C = Coupled(F, nsteps=nsteps)
    C.build(W, prec)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    return plan, F, C


def _cpl_by_block(bse, plan, spec, rho_cpl, q_range):
    """GPU coupling layout -> {(ik, ik2): (rvc [v][c'][NG], rcv [c][v'][NG])}."""
    nv, nc, w = spec.nv, spec.nc, spec.nv * spec.nc
    rd = rho_cpl.cpu().numpy()
    out, base = {}, 0
    for iq in q_range:
        blk, _ = bse.bse_pair_blocks(plan, 0, iq)
        ng = len(bse.bse_gvectors(plan, 0, iq, 1))
        nb = len(blk)
        for t, (ik, ik2) in enumerate(blk):
            rvc = rd[base + t * w: base + (t + 1) * w, :ng].reshape(nv, nc, ng)
            rcv = rd[base + nb * w + t * w: base + nb * w + (t + 1) * w, :ng].reshape(nc, nv, ng)
            out[(int(ik), int(ik2))] = (rvc, rcv)
        base += 2 * nb * w
    return out


@pytest.fixture(scope="module")
def cfg1_B(cfg1, cfg1_oracle):
    spec = cfg1.spec
    return cp.coupling_from_factors(spec, cfg1_oracle["rho_x"], cp.coupling_factors(spec, cfg1.gk, cfg1.coef), cfg1.W)


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("which", ["tiny", "cfg1"])
def test_coupling_pair_densities_every_block(bse, tiny_spec, cfg1, which):
    s = generate(tiny_spec) if which == "tiny" else cfg1
    spec = s.spec
    plan, F, C = _coupled(bse, s, 8)
    got = _cpl_by_block(bse, plan, spec, C.rho_cpl, range(spec.nkpt))
    worst = scale = 0.0
    for ik, ik2 in geo.upper_blocks(spec):
        _, rvc, rcv = cp.coupling_rho_block(spec, ik, ik2, s.gk, s.coef)
        gv, gc = got[(ik, ik2)]
        worst = max(worst, np.abs(gv - rvc).max(), np.abs(gc - rcv).max())
        scale = max(scale, np.abs(rvc).max(), np.abs(rcv).max())
    assert worst / scale < 1e-5


@pytest.mark.parametrize("prec,tol", [(0, 1e-5), (1, 1e-4)])
def test_coupling_matrix_matches_oracle_and_is_symmetric(bse, cfg1, cfg1_B, prec, tol):
    plan, F, C = _coupled(bse, cfg1, 8, prec=prec)
    B = C.Bm.cpu().numpy()
    assert np.array_equal(B, B.T)
    assert _relmax(B, cfg1_B) < tol


def test_coupling_q_chunked_equals_single_pass(bse, cfg1):
    _, _, C1 = _coupled(bse, cfg1, 8)
    _, _, C2 = _coupled(bse, cfg1, 8, qchunk=7)
    assert torch.equal(C1.Bm, C2.Bm)


def test_coupled_spectrum_matches_oracle(bse, cfg1, cfg1_oracle, cfg1_B):
    spec = cfg1.spec
    n = 100
    plan, F, C = _coupled(bse, cfg1, n)
    om = _dev(cfg1.omega, torch.float64)
    eps = C.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    assert int(C.steps_done.item()) == n
    A, B = F.H.cpu().numpy().astype(np.complex128), C.Bm.cpu().numpy().astype(np.complex128)
    ref, a, b, done, s2 = cp.eps2_lanczos(spec, A, B, F.P.cpu().numpy(), cfg1.omega, spec.eta, n)
    assert done == n
    bg = C.b.cpu().numpy()
    assert abs(bg[0] ** 2 - s2) < 1e-6 * s2
    assert np.abs(bg[1:] - b[1:]).max() < 1e-5 * b.max()
    assert np.abs(eps - ref).max() / ref.max() < 1e-5
    # end to end: the oracle's own A and B
    ref2 = cp.eps2_lanczos(spec, cfg1_oracle["H"], cfg1_B, cfg1_oracle["P"], cfg1.omega, spec.eta, n)[0]
    assert np.abs(eps - ref2).max() / ref2.max() < 1e-5
    # the coupling is visible: B = 0 moves eps_2 by far more than the tolerance
    ref0 = cp.eps2_lanczos(spec, A, 0 * B, F.P.cpu().numpy(), cfg1.omega, spec.eta, n)[0]
    assert np.abs(ref0 - ref).max() / ref.max() > 1e-4


def test_coupled_full_krylov_equals_direct_solve(bse, tiny_spec):
    s = generate(tiny_spec)
    spec = s.spec
    n = 2 * spec.dim
    plan, F, C = _coupled(bse, s, n)
    om = _dev(s.omega, torch.float64)
    eps = C.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    A, B = F.H.cpu().numpy().astype(np.complex128), C.Bm.cpu().numpy().astype(np.complex128)
    ref = cp.eps2_direct(spec, A, B, F.P.cpu().numpy(), s.omega, spec.eta)
    assert np.abs(eps - ref).max() / np.abs(ref).max() < 1e-5


def test_no_coupling_gives_resonant_minus_antiresonant(bse, cfg1):
    """B = 0 at the full Krylov dimension: C sum_l |P^H A_l|^2 [L(w - E_l) - L(w + E_l)] from eigh(A)."""
    spec = cfg1.spec
    n = 2 * spec.dim
    plan, F, C = _coupled(bse, cfg1, n)
    C.Bm.zero_()
    om = _dev(cfg1.omega, torch.float64)
    eps = C.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    e, v = np.linalg.eigh(F.H.cpu().numpy().astype(np.complex128))
    wts = np.abs(np.conj(F.P.cpu().numpy()) @ v) ** 2
    eta, w = spec.eta, cfg1.omega
    lor = lambda x: eta / (x * x + eta * eta)   # noqa: E731
    from oracle import spectrum as osp
    ref = osp.prefactor(spec) * (lor(w[:, None] - e[None, :]) - lor(w[:, None] + e[None, :])) @ wts
    assert np.abs(eps - ref).max() / ref.max() < 1e-5


def test_coupled_breakdown_two_energies(bse, cfg1):
    """Diagonal A with two distinct transition energies and B = 0: the Krylov space of s is spanned by
    the +-E pairs of the two energies, so the recursion stops after exactly four steps."""
    spec = cfg1.spec
    plan, F, C = _coupled(bse, cfg1, 40)
    e1 = np.where(np.arange(spec.dim) % 2 == 0, 0.2, 0.35)
    F.H.copy_(torch.diag(_dev(e1, torch.complex64)))
    C.Bm.zero_()
    om = _dev(cfg1.omega, torch.float64)
    eps = C.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    assert int(C.steps_done.item()) == 4
    P = F.P.cpu().numpy()
    eta, w = spec.eta, cfg1.omega
    lor = lambda x: eta / (x * x + eta * eta)   # noqa: E731
    from oracle import spectrum as osp
    ref = osp.prefactor(spec) * ((lor(w[:, None] - e1[None, :]) - lor(w[:, None] + e1[None, :])) @ (np.abs(P) ** 2))
    assert np.abs(eps - ref).max() / ref.max() < 1e-5


def test_unstable_system_reports_indefinite(bse, cfg1):
    """A = 0.1 I, B = 0.5 I: M = F H2 has eigenvalues 0.1 -+ 0.5.  With a real P the first M-norm is
    positive and the second negative: the recursion stops after one step with BSE_ERR_INDEFINITE."""
    spec = cfg1.spec
    plan, F, C = _coupled(bse, cfg1, 20)
    eye = torch.eye(spec.dim, dtype=torch.complex64, device="cuda")
    F.H.copy_(0.1 * eye)
    C.Bm.copy_(0.5 * eye)
    F.P.copy_(_dev(np.linspace(1.0, 2.0, spec.dim), torch.complex128))
    om = _dev(cfg1.omega, torch.float64)
    C.spectrum(om, spec.eta)
    with pytest.raises(bse.BseError) as ei:
        bse.bse_status_read(plan)
    assert ei.value.code == bse.BSE_ERR_INDEFINITE
    assert int(C.steps_done.item()) == 1
    # the plan stays usable
    plan2, F2, C2 = _coupled(bse, cfg1, 10)
    C2.spectrum(om, spec.eta)
    bse.bse_status_read(plan2)
    assert int(C2.steps_done.item()) == 10


def _oracle_cpl_block(spec, s, ik, ik2):
    g0 = geo.sphere(spec, (0, 0, 0))
    vb, cb = list(range(spec.nv)), list(range(spec.nv, spec.nb))
    rx = op.rho_corr(spec, ik, ik, vb, cb, g0, s.gk, s.coef).reshape(spec.nv * spec.nc, -1)
    rx2 = op.rho_corr(spec, ik2, ik2, vb, cb, g0, s.gk, s.coef).reshape(spec.nv * spec.nc, -1)
    mi = cp.minus_g_index(spec)
    bx = ok.norm_factor(spec) * (np.conj(rx) * ok.coulomb_bar(spec)[None, :]) @ np.conj(rx2[:, mi]).T
    iq, rvc, rcv = cp.coupling_rho_block(spec, ik, ik2, s.gk, s.coef)
    blk = 2.0 * bx - cp.coupling_direct_block(spec, rvc, rcv, ok.w_of_q(spec, s.W, iq))
    if ik == ik2:
        blk = 0.5 * (blk + blk.T)
    return blk


def test_coupled_fcc8_full_size(bse):
    """fcc 8x8x8 3v4c (dim 6144), the bench workload with the bench's q chunks: sampled blocks of B against
    the oracle, and the 600-step coupled recursion against the oracle's FP64 recursion on the same A, B."""
    spec = config_spec("fcc_8x8x8_3v4c")
    s = generate(spec, wdtype=np.complex64)
    n = 600
    plan, F, C = _coupled(bse, s, n, qchunk=64)
    B = C.Bm.cpu().numpy()
    assert np.array_equal(B, B.T)
    rng = np.random.default_rng(11)
    nvc = spec.nv * spec.nc
    blocks = [(0, 0), (0, 511), (37, 200), (300, 300)] + [tuple(sorted(rng.integers(0, spec.nkpt, 2))) for _ in range(4)]
    for ik, ik2 in blocks:
        ref = _oracle_cpl_block(spec, s, ik, ik2)
        got = B[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc]
        assert np.abs(got - ref).max() < 1e-5 * np.abs(B).max(), (ik, ik2)
    om = _dev(s.omega, torch.float64)
    eps = C.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    assert int(C.steps_done.item()) == n
    A = F.H.cpu().numpy().astype(np.complex128)
    ref, a, b, done, s2 = cp.eps2_lanczos(spec, A, B.astype(np.complex128), F.P.cpu().numpy(), s.omega, spec.eta, n)
    assert np.abs(eps - ref).max() / ref.max() < 1e-5
    assert np.abs(C.b.cpu().numpy()[1:] - b[1:]).max() < 1e-5 * b.max()
