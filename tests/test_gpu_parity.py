"""CUDA path against the CPU oracle (through the C ABI).

Tolerances (FP32 path): pair densities and H within 1e-5 of their max entry;
eps_2 within 1e-5 of its peak.  The FP32 rounding of H alone moves eigenvalues
by ~1e-7 |H|, i.e. eps_2 by ~1e-7 |H|/eta relative near a peak, well inside 1e-5
for eta = 0.1 eV and |H| ~ 0.6 Ha.
"""
import numpy as np
import pytest

from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp
from synth import SystemSpec, generate

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


def _forward(bse, sysd, nsteps, nw=None, qchunk=None, keep=True, prec=0, delta=None, method=None):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = sysd.spec
    plan = bse.Plan([spec])
    if method is not None:          # "fft" or "correlation" pair densities (default: the planner's choice)
        variants, _ = bse.bse_pair_variants(plan, 0)
        v = next(x for x in variants if (x["rows"] == 0) == (method == "correlation"))
        bse.bse_set_pair_variant(plan, 0, v["index"])
    nw = len(sysd.omega) if nw is None else nw
    F = Forward(plan, 0, nsteps=nsteps, nw=nw, qchunk=qchunk, keep_rho_dir=keep)
    coef = _dev(sysd.coef, torch.complex64)
    en = _dev(sysd.energies, torch.float64)
    W = _dev(sysd.W, torch.complex64)
    F.build(coef, en, W, spec.delta if delta is None else delta, prec)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    return plan, F


def _rho_dir_by_block(bse, plan, spec, rho_dir):
    """GPU rho_dir layout -> {(ik, ik2): (rv [v][v'][NG], rc [c][c'][NG])}."""
    nv, nc = spec.nv, spec.nc
    out = {}
    base = 0
    rd = rho_dir.cpu().numpy()
    for iq in range(spec.nkpt):
        blk, _ = bse.bse_pair_blocks(plan, 0, iq)
        ng = len(bse.bse_gvectors(plan, 0, iq, 1))
        nb = len(blk)
        for t, (ik, ik2) in enumerate(blk):
            rv = rd[base + t * nv * nv: base + (t + 1) * nv * nv, :ng].reshape(nv, nv, ng)
            rc = rd[base + nb * nv * nv + t * nc * nc: base + nb * nv * nv + (t + 1) * nc * nc, :ng].reshape(nc, nc, ng)
            out[(int(ik), int(ik2))] = (rv, rc)
        base += nb * (nv * nv + nc * nc)
    return out


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("method", ["correlation", "fft"])
def test_exchange_pair_densities_and_dipole(bse, cfg1, cfg1_oracle, method):
    plan, F = _forward(bse, cfg1, 100, method=method)
    rx = F.rho_x.cpu().numpy()[:, :113]
    assert _relmax(rx, cfg1_oracle["rho_x"]) < 1e-5
    assert _relmax(F.P.cpu().numpy(), cfg1_oracle["P"]) < 1e-6


@pytest.mark.parametrize("method", ["correlation", "fft"])
def test_direct_pair_densities_every_block(bse, cfg1, cfg1_oracle, method):
    plan, F = _forward(bse, cfg1, 100, method=method)
    got = _rho_dir_by_block(bse, plan, cfg1.spec, F.rho_dir)
    scale = max(np.abs(f[3]).max() for f in cfg1_oracle["factors"])
    worst = 0.0
    for ik, ik2, iq, rv, rc in cfg1_oracle["factors"]:
        gv, gc = got[(ik, ik2)]
        worst = max(worst, np.abs(gv - rv).max(), np.abs(gc - rc).max())
    assert worst / scale < 1e-5


def test_hamiltonian_matches_oracle_and_is_hermitian(bse, cfg1, cfg1_oracle):
    plan, F = _forward(bse, cfg1, 100)
    H = F.H.cpu().numpy()
    assert np.array_equal(H, H.conj().T)
    assert _relmax(H, cfg1_oracle["H"]) < 1e-5
    # the kernel part alone (off-diagonal), relative to its own scale
    Href = cfg1_oracle["H"]
    off = ~np.eye(576, dtype=bool)
    assert np.abs(H - Href)[off].max() / np.abs(Href[off]).max() < 1e-5


def test_hamiltonian_q_chunked_equals_single_pass(bse, cfg1):
    _, F1 = _forward(bse, cfg1, 100)
    _, F2 = _forward(bse, cfg1, 100, qchunk=7, keep=False)
    assert torch.equal(F1.H, F2.H)


def test_spectrum_matches_oracle_haydock(bse, cfg1, cfg1_oracle):
    spec = cfg1.spec
    plan, F = _forward(bse, cfg1, 100)
    om = _dev(cfg1.omega, torch.float64)
    eps = F.spectrum(om, spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    assert int(F.steps_done.item()) == 100
    ref, a, b, _ = osp.eps2_haydock(spec, cfg1_oracle["H"], cfg1_oracle["P"], cfg1.omega, spec.eta, 100)
    assert np.abs(eps - ref).max() / ref.max() < 1e-5
    ab = F.ab.cpu().numpy()
    # the 100-step coefficients move by ~5e-6 of their maximum when the oracle's own H is stored in FP32
    # (1.6e-5 under a random Hermitian change of 3e-8 max|H|): an FP32 pipeline is held to 10x that floor
    a32, b32, _, _ = osp.haydock(cfg1_oracle["H"].astype(np.complex64).astype(np.complex128), cfg1_oracle["P"], 100)
    fa = np.abs(a32 - a).max() / np.abs(a).max()
    fb = np.abs(b32 - b).max() / np.abs(b).max()
    ea = np.abs(ab[:100] - a).max() / np.abs(a).max()
    eb = np.abs(ab[100:] - b).max() / np.abs(b).max()
    print(f"Haydock coefficients vs the oracle: a {ea:.2e} (FP32-storage floor {fa:.2e}), "
          f"b {eb:.2e} (floor {fb:.2e}); eps_2 {np.abs(eps - ref).max() / ref.max():.2e}")
    assert ea < max(1e-5, 10.0 * fa)
    assert eb < max(1e-5, 10.0 * fb)


def test_spectrum_full_krylov_equals_dense_eig(bse, cfg1, cfg1_oracle):
    spec = cfg1.spec
    plan, F = _forward(bse, cfg1, 576)
    om = _dev(cfg1.omega, torch.float64)
    eps = F.spectrum(om, spec.eta, nsteps=576).cpu().numpy()
    ref = osp.eps2_dense(spec, cfg1_oracle["H"], cfg1_oracle["P"], cfg1.omega, spec.eta)
    assert np.abs(eps - ref).max() / ref.max() < 1e-5


def test_apply_h_matches_host_product(bse, cfg1):
    plan, F = _forward(bse, cfg1, 100)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, 576)) + 1j * rng.standard_normal((3, 576))
    Xd = _dev(X, torch.complex128)
    Y = torch.empty_like(Xd)
    bse.bse_apply_H(plan, 0, F.H, Xd, Y)
    ref = (F.H.cpu().numpy().astype(np.complex128) @ X.T).T
    assert _relmax(Y.cpu().numpy(), ref) < 1e-6


@pytest.mark.parametrize("nk,nv,nc", [(3, 1, 1), (2, 1, 3), (3, 2, 1)])
def test_ragged_small_systems(bse, nk, nv, nc):
    """Odd dimensions (27, 9*... ), single bands, one-block rows: full pipeline vs oracle."""
    spec = SystemSpec(f"t{nk}{nv}{nc}", "fcc", 10.0, 0.0, (nk, nk, nk), nv, nc, 1.0, (8, 8, 8), "3d", nsteps=8, nw=120)
    s = generate(spec)
    n = min(8, spec.dim)
    plan, F = _forward(bse, s, n)
    om = _dev(s.omega, torch.float64)
    eps = F.spectrum(om, spec.eta, nsteps=n).cpu().numpy()
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    assert _relmax(F.H.cpu().numpy(), H) < 1e-5
    ref = osp.eps2_haydock(spec, H, P, s.omega, spec.eta, n)[0]
    assert np.abs(eps - ref).max() / ref.max() < 1e-5


def test_breakdown_reports_fewer_steps(bse):
    """nsteps = dim on a 27-dim system: the recursion matches the oracle's step count and spectrum.
    With the kernel off (rho_x = 0, no direct term) H is diagonal with two distinct transition
    energies: the Krylov space of P closes after two vectors (up to the FP32 rounding of the
    matrix-vector product, ~1e-7 |H v|, below the 1e-6 breakdown threshold), so the recursion must
    stop after exactly two steps and reproduce the closed-form independent-particle spectrum."""
    spec = SystemSpec("brk", "fcc", 10.0, 0.0, (3, 3, 3), 1, 1, 1.0, (8, 8, 8), "3d", nsteps=27, nw=100)
    s = generate(spec)
    e = s.energies.copy()
    e[:, 0] = -0.1
    e[:, 1] = np.where(np.arange(27) % 2 == 0, 0.2, 0.3)     # two distinct transition energies
    s.energies = e
    s.W[:] = 0.0
    plan, F = _forward(bse, s, 27)
    om = _dev(s.omega, torch.float64)
    eps = F.spectrum(om, spec.eta, nsteps=27).cpu().numpy()
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    ref, _, _, done = osp.eps2_haydock(spec, H, P, s.omega, spec.eta, 27)
    assert int(F.steps_done.item()) == done
    assert np.abs(eps - ref).max() / ref.max() < 1e-5
    # kernel off
    e1 = s.energies
    en = _dev(e1, torch.float64)
    F.rho_x.zero_()
    bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT | bse.BSE_BK_MIRROR, F.rho_x, None, 0, 0, None, en, spec.delta,
                         bse.BSE_PREC_FP32, F.H, None)
    eps0 = F.spectrum(om, spec.eta, nsteps=27).cpu().numpy()
    bse.bse_status_read(plan)
    assert int(F.steps_done.item()) == 2
    de = ok.transition_energies(spec, e1, spec.delta)
    ip = osp.eps2_independent(spec, de, P, s.omega, spec.eta)
    assert np.abs(eps0 - ip).max() / ip.max() < 1e-5


def test_error_returns_on_a_device_plan(bse, tiny_spec):
    """Invalid ranges, step counts and workspaces are refused before any launch."""
    from paper_1206_3518_gb300.pipeline import Forward
    plan = bse.Plan([tiny_spec])
    F = Forward(plan, 0, nsteps=8, nw=16)
    om = torch.zeros(16, dtype=torch.float64, device="cuda")
    cases = [
        (lambda: bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, 3, 3,
                                        F.ws_pair), bse.BSE_ERR_ARG),
        (lambda: bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, 0, 1,
                                        F.ws_pair[:16]), bse.BSE_ERR_WORKSPACE),
        (lambda: bse.bse_spectrum(plan, 0, F.H, F.P, 0, om, 0.01, F.eps2[:16], F.ab, F.steps_done, F.ws_spec),
         bse.BSE_ERR_ARG),
        (lambda: bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT | bse.BSE_BK_MIRROR, None, F.rho_dir, 0, 1,
                                      F.rho_x, None, 0.0, bse.BSE_PREC_FP32, F.H, F.ws_kernel), bse.BSE_ERR_ARG),
        (lambda: bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, 0, 1, F.rho_x, None, 0.0, 7,
                                      F.H, F.ws_kernel), bse.BSE_ERR_ARG),
    ]
    for call, code in cases:
        with pytest.raises(bse.BseError) as err:
            call()
        assert err.value.code == code
    bse.bse_status_read(plan)


def test_ritz_pairs_match_oracle_and_spectrum(bse, cfg1):
    """bse_ritz on the GPU's own Haydock coefficients: Ritz values and weights against the oracle's
    tridiagonal eigen-solve (FP64 both, 1e-10), the pole sum reproduces the GPU eps_2, and at full
    Krylov dimension the bright Ritz pairs are the eigenpairs of H (exciton energies, strengths)."""
    spec = cfg1.spec
    om = _dev(cfg1.omega, torch.float64)
    for n in (100, 576):
        plan, F = _forward(bse, cfg1, n)
        eps = F.spectrum(om, spec.eta, nsteps=n).cpu().numpy()
        theta = torch.zeros(n, dtype=torch.float64, device="cuda")
        w = torch.zeros_like(theta)
        ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_RITZ, n) // 8, dtype=torch.float64, device="cuda")
        bse.bse_ritz(F.ab, F.steps_done, n, theta, w, ws)
        bse.bse_status_read(plan)
        done = int(F.steps_done.item())
        ab = F.ab.cpu().numpy()
        th_ref, w_ref = osp.ritz(ab[:done], ab[n:n + done])
        th, wg = theta.cpu().numpy()[:done], w.cpu().numpy()[:done]
        assert np.abs(th - th_ref).max() < 1e-10 * np.abs(th_ref).max()
        assert np.abs(wg - w_ref).max() < 1e-10
        P = F.P.cpu().numpy()
        z = cfg1.omega + 1j * spec.eta
        pole = -osp.prefactor(spec) * np.vdot(P, P).real * (wg[None, :] / (z[:, None] - th[None, :])).sum(1).imag
        assert np.abs(pole - eps).max() < 1e-9 * eps.max()
        if n == 576:
            e, v = np.linalg.eigh(F.H.cpu().numpy().astype(np.complex128))
            wt = np.abs(np.conj(P) @ v) ** 2 / np.vdot(P, P).real
            bright = wg > 1e-4
            assert bright.sum() > 20
            # a Ritz weight is a squared eigenvector component of a recursion with FP32 products of H:
            # its error grows like 1e-7 |H| / (gap to the nearest other eigenvalue), ~1e-3 relative for
            # gaps of 1e-4 Ha; eigenvalues closer than 1e-6 appear as one Ritz value (their weights sum)
            for t, x in zip(th[bright], wg[bright]):
                cl = np.abs(e - t) < 1e-6
                assert cl.any() and abs(wt[cl].sum() - x) < 1e-3 * x
