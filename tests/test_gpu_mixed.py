"""BF16 hi/lo split-complex contractions on tcgen05 (precision BSE_PREC_BF16X3) against FP32 and the oracle.

Each operand x = hi + lo in BF16; three products per pair (hi.hi, hi.lo, lo.hi) accumulate in FP32,
so each product carries ~2^-16 relative error: kernel entries within 1e-4 of the largest kernel
entry, eps_2 within 1e-3 of its peak (the mixed-precision tolerance).
"""
import numpy as np
import pytest

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


def _build(bse, s, prec, nsteps):
    from paper_1206_3518_gb300.pipeline import Forward
    plan = bse.Plan([s.spec])
    F = Forward(plan, 0, nsteps=nsteps, nw=len(s.omega))
    F.build(_dev(s.coef, torch.complex64), _dev(s.energies, torch.float64), _dev(s.W, torch.complex64),
            s.spec.delta, prec)
    eps = F.spectrum(_dev(s.omega, torch.float64), s.spec.eta).cpu().numpy()
    bse.bse_status_read(plan)
    return F.H.cpu().numpy(), eps


def test_bf16x3_kernel_and_spectrum_cfg1(bse, cfg1, cfg1_oracle):
    spec = cfg1.spec
    H32, e32 = _build(bse, cfg1, bse.BSE_PREC_FP32, 100)
    Hbf, ebf = _build(bse, cfg1, bse.BSE_PREC_BF16X3, 100)
    off = ~np.eye(spec.dim, dtype=bool)
    kscale = np.abs(H32[off]).max()
    assert np.abs(Hbf - H32)[off].max() / kscale < 1e-4
    assert np.array_equal(Hbf, Hbf.conj().T)
    ref = osp.eps2_haydock(spec, cfg1_oracle["H"], cfg1_oracle["P"], cfg1.omega, spec.eta, 100)[0]
    assert np.abs(ebf - ref).max() / ref.max() < 1e-3
    Koracle = cfg1_oracle["H"][off]
    assert np.abs(Hbf[off] - Koracle).max() / np.abs(Koracle).max() < 1e-4


def test_bf16x3_with_conduction_side_operand(bse):
    """nc^2 < nv^2: the W product is taken on the conduction side."""
    spec = SystemSpec("side_c", "fcc", 10.0, 0.0, (3, 3, 3), 3, 2, 1.0, (8, 8, 8), "3d", nsteps=20, nw=150)
    s = generate(spec)
    Hbf, ebf = _build(bse, s, bse.BSE_PREC_BF16X3, 20)
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    off = ~np.eye(spec.dim, dtype=bool)
    assert np.abs(Hbf - H)[off].max() / np.abs(H[off]).max() < 1e-4
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    ref = osp.eps2_haydock(spec, H, P, s.omega, spec.eta, 20)[0]
    assert np.abs(ebf - ref).max() / ref.max() < 1e-3
