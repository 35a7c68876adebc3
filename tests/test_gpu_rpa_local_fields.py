"""Spectrum with local fields in the random-phase approximation, Tamm-Dancoff form.

With the screened direct term left out, H = diag(e_c + Delta - e_v) + 2 K^x is the TDA form of
the RPA response with local fields (the irreducible chi-bar of Eq. epsilon_chi_bar with the
short-range exchange Vbar only).  The GPU path is the BSE path with the direct term skipped
(bse_build_kernel with BSE_BK_INIT | BSE_BK_MIRROR); the oracle builds the same Hamiltonian from its own
pair densities and takes the spectrum by dense diagonalisation (Haydock with nsteps = dim is
exact).
"""
import numpy as np
import pytest

from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp

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


def test_exchange_only_spectrum_matches_oracle(bse, cfg1, cfg1_oracle):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = cfg1.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.dim, nw=spec.nw)
    dev = lambda x, t: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=t)  # noqa: E731
    en = dev(cfg1.energies, torch.float64)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, dev(cfg1.coef, torch.complex64), en,
                           F.rho_x, F.P, None, 0, 0, F.ws_pair)
    bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT | bse.BSE_BK_MIRROR, F.rho_x, None, 0, 0, None, en, spec.delta,
                         bse.BSE_PREC_FP32, F.H, None)
    Hg = F.H.cpu().numpy()
    assert np.array_equal(Hg, Hg.conj().T)
    Href = np.diag(ok.transition_energies(spec, cfg1.energies, spec.delta)) + 2.0 * ok.exchange_kernel(
        spec, cfg1_oracle["rho_x"])
    off = ~np.eye(spec.dim, dtype=bool)
    assert np.abs(Hg - Href)[off].max() / np.abs(Href[off]).max() < 1e-5
    P = op.dipole(spec, cfg1.gk, cfg1.coef, cfg1.energies)
    ref = osp.eps2_dense(spec, Href, P, cfg1.omega, spec.eta)
    eps = F.spectrum(dev(cfg1.omega, torch.float64), spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    assert np.abs(eps - ref).max() / ref.max() < 1e-5
    # local fields move weight relative to the independent-particle spectrum
    ip = osp.eps2_independent(spec, ok.transition_energies(spec, cfg1.energies, spec.delta), P, cfg1.omega, spec.eta)
    assert np.abs(ref - ip).max() > 1e-3 * ip.max()


@pytest.mark.parametrize("name", ["fcc_4x4x4_3v3c", "side_3v2c"])
def test_exchange_kernel_on_tensor_cores(bse, cfg1, cfg1_oracle, name):
    """diag + 2 K^x as the BF16x3 tcgen05 Gram product (BSE_BK_INIT with BSE_PREC_BF16X3 and a workspace):
    within 1e-4 of the largest kernel entry of the oracle's exchange-only H (BF16x3 ~2^-16 per product),
    the diagonal transition energies exact to FP32; and the FP32 route without a workspace unchanged."""
    from paper_1206_3518_gb300.pipeline import Forward
    from synth import SystemSpec, generate
    if name == "side_3v2c":
        s = generate(SystemSpec(name, "fcc", 10.0, 0.0, (3, 3, 3), 3, 2, 1.0, (8, 8, 8), "3d", nsteps=20, nw=150))
        rho_ref = op.exchange_rho(s.spec, s.gk, s.coef)
    else:
        s, rho_ref = cfg1, cfg1_oracle["rho_x"]
    spec = s.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=10, nw=10)
    dev = lambda x, t: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=t)  # noqa: E731
    en = dev(s.energies, torch.float64)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, dev(s.coef, torch.complex64), en,
                           F.rho_x, F.P, None, 0, 0, F.ws_pair)
    bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT | bse.BSE_BK_MIRROR, F.rho_x, None, 0, 0, None, en, spec.delta,
                         bse.BSE_PREC_BF16X3, F.H, F.ws_kernel)
    bse.bse_status_read(plan)
    Hg = F.H.cpu().numpy().astype(np.complex128)
    Href = np.diag(ok.transition_energies(spec, s.energies, spec.delta)) + 2.0 * ok.exchange_kernel(spec, rho_ref)
    off = ~np.eye(spec.dim, dtype=bool)
    err = np.abs(Hg - Href)[off].max() / np.abs(Href[off]).max()
    derr = np.abs(np.diag(Hg) - np.diag(Href)).max() / np.abs(np.diag(Href)).max()
    bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT | bse.BSE_BK_MIRROR, F.rho_x, None, 0, 0, None, en, spec.delta,
                         bse.BSE_PREC_FP32, F.H, None)
    err32 = np.abs(F.H.cpu().numpy() - Href)[off].max() / np.abs(Href[off]).max()
    print(f"{name}: tensor-core exchange kernel vs the oracle {err:.2e} of the largest kernel entry (diagonal "
          f"{derr:.2e}); FP32 route {err32:.2e}")
    assert err < 1e-4 and derr < 1e-5 and err32 < 1e-5
    assert np.array_equal(Hg, Hg.conj().T)
