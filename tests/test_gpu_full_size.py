"""Parity at the workloads' full sizes (sampled outputs the oracle computes one by one, and
properties that hold at any size), plus full parity for every compiled grid variant on small cells."""
import math

import numpy as np
import pytest

from oracle import geometry as geo
from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp
from synth import SystemSpec, config_spec, generate, slab_batch_specs

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


def _exchange_rows(spec, s, ik):
    """rho_x rows of k (S = (k, v, c)) from the oracle's plane-wave correlation."""
    g0 = geo.sphere(spec, (0, 0, 0))
    r = op.rho_corr(spec, ik, ik, list(range(spec.nv)), list(range(spec.nv, spec.nb)), g0, s.gk, s.coef)
    return r.reshape(spec.nv * spec.nc, -1)


def _oracle_block(spec, s, ik, ik2, delta):
    """H block (k, k') from the oracle: diag + 2 K^x - K^d, computed for this block only."""
    nvc = spec.nv * spec.nc
    v = ok.coulomb_bar(spec)
    rx = _exchange_rows(spec, s, ik)
    rx2 = _exchange_rows(spec, s, ik2)
    kx = ok.norm_factor(spec) * (np.conj(rx) * v[None, :]) @ rx2.T
    iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
    kd = ok.direct_block(spec, rv, rc, ok.w_of_q(spec, s.W, iq))
    blk = 2.0 * kx - kd
    if ik == ik2:
        blk = blk + np.diag(ok.transition_energies(spec, s.energies, delta)[ik * nvc:(ik + 1) * nvc])
        blk = 0.5 * (blk + blk.conj().T)
    return blk, (iq, rv, rc)


def _sampled_parity(bse, s, qchunk, nsample, seed, tol=1e-5):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = s.spec
    plan = bse.Plan([spec])
    inf = plan.info(0)
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=len(s.omega), qchunk=qchunk)
    coef = _dev(s.coef, torch.complex64)
    en = _dev(s.energies, torch.float64)
    W = _dev(s.W, torch.complex64)
    F.build(coef, en, W, spec.delta)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    rng = np.random.default_rng(seed)
    nvc = spec.nv * spec.nc
    rxg = F.rho_x.cpu().numpy()[:, :inf["ng0"]]
    for ik in rng.integers(0, spec.nkpt, 8):
        ref = _exchange_rows(spec, s, ik)
        assert np.abs(rxg[ik * nvc:(ik + 1) * nvc] - ref).max() / np.abs(ref).max() < tol
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    assert np.abs(F.P.cpu().numpy() - P).max() / np.abs(P).max() < 1e-6
    blocks = [(0, 0)] + [tuple(sorted(rng.integers(0, spec.nkpt, 2))) for _ in range(nsample)]
    worst = 0.0
    hscale = 0.0
    for ik, ik2 in blocks:
        ref, _ = _oracle_block(spec, s, ik, ik2, spec.delta)
        got = F.H[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc].cpu().numpy()
        mir = F.H[ik2 * nvc:(ik2 + 1) * nvc, ik * nvc:(ik + 1) * nvc].cpu().numpy()
        assert np.array_equal(mir, got.conj().T)
        off = ~np.eye(nvc, dtype=bool) if ik == ik2 else np.ones((nvc, nvc), bool)
        worst = max(worst, np.abs(got - ref)[off].max())
        hscale = max(hscale, np.abs(ref[off]).max())
    assert worst / hscale < tol
    return plan, F, P


def _sum_rule(bse, plan, F, spec, P, nsteps):
    """Zeroth moment: int eps_2 dw over the real line = pi C |P|^2 for any number of steps."""
    w = np.linspace(-4.0, 4.0, 200001)
    om = _dev(w, torch.float64)
    from paper_1206_3518_gb300.pipeline import Forward  # noqa: F401
    eps = torch.empty(len(w), dtype=torch.float64, device="cuda")
    ab = torch.empty(2 * nsteps, dtype=torch.float64, device="cuda")
    done = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_SPECTRUM, nsteps) // 8 + 1, dtype=torch.complex64,
                     device="cuda")
    eta = 0.02
    bse.bse_spectrum(plan, 0, F.H, F.P, nsteps, om, eta, eps, ab, done, ws)
    bse.bse_status_read(plan)
    e = eps.cpu().numpy()
    assert e.min() > -1e-12 * e.max()
    integral = np.sum(0.5 * (e[1:] + e[:-1]) * np.diff(w))
    c = osp.prefactor(spec) * np.vdot(P, P).real
    # Lorentzian tails beyond the window carry about 2 eta/(pi * 4 Ha) of the weight
    assert abs(integral - math.pi * c) / (math.pi * c) < 1e-2
    a = ab.cpu().numpy()
    assert int(done.item()) == nsteps and np.all(a[nsteps + 1:nsteps + nsteps] > 0)


def test_bench_workload_fcc8_sampled(bse):
    """fcc 8x8x8 3v4c (dim 6144) in the launch configuration bench.py times (all q in one chunk)."""
    s = generate(config_spec("fcc_8x8x8_3v4c"), wdtype=np.complex64)
    plan, F, P = _sampled_parity(bse, s, None, 24, 7)
    _sum_rule(bse, plan, F, s.spec, P, 300)


def test_fcc12_full_size_sampled(bse):
    """fcc 12x12x12 4v4c (dim 27648, 48^3 grid) streamed in q chunks.

    Kernel sums run over up to 531 x 531 G pairs in FP32; the measured error of the kernel
    entries is 1.3e-5 of the largest one, bounded here by 1e-4 (this workload's own bound is
    1e-3 on the spectrum).
    """
    s = generate(config_spec("fcc_12x12x12_4v4c"), wdtype=np.complex64)
    plan, F, P = _sampled_parity(bse, s, 96, 12, 11, tol=1e-4)
    _sum_rule(bse, plan, F, s.spec, P, 60)


@pytest.mark.parametrize("method", ["correlation", "fft"])
@pytest.mark.parametrize("name", ["g48", "hex", "hex_dirac"])
def test_grid_variant_full_parity(bse, name, method):
    """The plane-wave correlation kernel and the first compiled FFT variant of each grid against the full
    oracle build and Haydock on a small cell."""
    from paper_1206_3518_gb300.pipeline import Forward
    if name == "g48":
        spec = config_spec("fcc_12x12x12_4v4c").replace(name="g48", nk=(2, 2, 2), nsteps=20, nw=200)
    else:
        base = slab_batch_specs(0)[0 if name == "hex_dirac" else 5]
        spec = base.replace(name=name, nk=(6, 6, 1), nsteps=20, nw=200)
    s = generate(spec)
    plan = bse.Plan([spec])
    variants, _ = bse.bse_pair_variants(plan, 0)
    v = next(x for x in variants if (x["rows"] == 0) == (method == "correlation"))
    bse.bse_set_pair_variant(plan, 0, v["index"])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    F.build(_dev(s.coef, torch.complex64), _dev(s.energies, torch.float64), _dev(s.W, torch.complex64), spec.delta)
    eps = F.spectrum(_dev(s.omega, torch.float64), spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    Pv = op.dipole(spec, s.gk, s.coef, s.energies)
    Hg = F.H.cpu().numpy()
    assert np.abs(Hg - H).max() / np.abs(H).max() < 1e-5
    off = ~np.eye(spec.dim, dtype=bool)
    assert np.abs(Hg - H)[off].max() / np.abs(H[off]).max() < 1e-5
    ref = osp.eps2_haydock(spec, H, Pv, s.omega, spec.eta, spec.nsteps)[0]
    # floor set by storing H in FP32 (from the oracle alone): these cells' eps_2 moves by ~2e-5 of its
    # peak under a random Hermitian change of 1e-7 max|H|, so an FP32 pipeline is held to 10x that floor
    r32 = osp.eps2_haydock(spec, H.astype(np.complex64).astype(np.complex128), Pv, s.omega, spec.eta, spec.nsteps)[0]
    floor = np.abs(r32 - ref).max() / ref.max()
    assert np.abs(eps - ref).max() / ref.max() < max(1e-5, 10.0 * floor)


def test_fcc12_mixed_precision_sampled(bse):
    """fcc 12x12x12 4v4c (dim 27648): BF16x3 tensor-core build against the oracle on sampled blocks
    (max and mean relative error of the kernel entries) and its eps_2 against the FP32 build's (the
    FP32 build is itself checked against the oracle above); tolerance 1e-3 of the eps_2 peak."""
    from paper_1206_3518_gb300.pipeline import Forward
    s = generate(config_spec("fcc_12x12x12_4v4c"), wdtype=np.complex64)
    spec = s.spec
    plan = bse.Plan([spec])
    nsteps = 60
    F = Forward(plan, 0, nsteps=nsteps, nw=len(s.omega), qchunk=96)
    coef, en, W = _dev(s.coef, torch.complex64), _dev(s.energies, torch.float64), _dev(s.W, torch.complex64)
    om = _dev(s.omega, torch.float64)
    F.build(coef, en, W, spec.delta, bse.BSE_PREC_FP32)
    e32 = F.spectrum(om, spec.eta, nsteps).cpu().numpy().copy()
    F.build(coef, en, W, spec.delta, bse.BSE_PREC_BF16X3)
    ebf = F.spectrum(om, spec.eta, nsteps).cpu().numpy().copy()
    bse.bse_status_read(plan)
    assert np.abs(ebf - e32).max() / e32.max() < 1e-3
    rng = np.random.default_rng(12)
    nvc = spec.nv * spec.nc
    errs, scale = [], 0.0
    for ik, ik2 in [(0, 0)] + [tuple(sorted(rng.integers(0, spec.nkpt, 2))) for _ in range(12)]:
        ref, _ = _oracle_block(spec, s, ik, ik2, spec.delta)
        got = F.H[ik * nvc:(ik + 1) * nvc, ik2 * nvc:(ik2 + 1) * nvc].cpu().numpy()
        off = ~np.eye(nvc, dtype=bool) if ik == ik2 else np.ones((nvc, nvc), bool)
        errs.append(np.abs(got - ref)[off].ravel())
        scale = max(scale, np.abs(ref[off]).max())
    err = np.concatenate(errs) / scale
    print(f"fcc12 BF16x3 kernel entries: max {err.max():.2e}, mean {err.mean():.2e} of the largest; "
          f"eps_2 vs FP32 {np.abs(ebf - e32).max() / e32.max():.2e}")
    assert err.max() < 1e-3 and err.mean() < 1e-4
