"""Differentiation workload: fcc 8x8x8 3v4c (dim 6144), loss over 512 frequencies, through the C ABI.

L = sum_w (1/512) (eps_2(w) - target(w))^2 with the target from the same system at Delta = 1.0 eV and
eps_inf = 9 (same random draws).  The adjoint (Lanczos recomputed, Krylov resolvent) is checked
against finite differences of the GPU forward: Delta by the exact rigid shift
eps_2(w; Delta + h) = eps_2(w - h; Delta), W along two Hermitian, reciprocal directions (each
summing the gradient over every entry).  Central differences at h and 2h are combined
(Richardson) to cancel the h^2 term.  The Krylov gradient is the exact resolvent gradient only
once the recursion has converged at eta, so the run uses 2400 steps (the change of eps_2 from
1200 to 2400 steps is checked to be small).
"""
import numpy as np
import pytest

from synth import config_spec, generate
from synth.systems import EV

from gradcheck import richardson_fd, w_directions

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NSTEPS = 2400


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


def test_adjoint_matches_finite_differences_fcc8_512w(bse):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = config_spec("fcc_8x8x8_3v4c").replace(nw=512)
    s = generate(spec, wdtype=np.complex64)
    tspec = spec.replace(eps_inf=9.0, delta=1.0 * EV)
    st = generate(tspec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=NSTEPS, nw=spec.nw, keep_rho_dir=True)
    coef, en = _dev(s.coef, torch.complex64), _dev(s.energies, torch.float64)
    W = _dev(s.W, torch.complex64)
    om = _dev(s.omega, torch.float64)
    F.build(coef, en, _dev(st.W, torch.complex64), tspec.delta)
    target = F.spectrum(om, spec.eta, NSTEPS).cpu().numpy().copy()
    F.build(coef, en, W, spec.delta)
    half = F.spectrum(om, spec.eta, NSTEPS // 2).cpu().numpy().copy()
    wgt = np.full(spec.nw, 1.0 / spec.nw)

    def loss(Wd=None, shift=0.0):
        if Wd is not None:
            F.build(coef, en, Wd, spec.delta)
        e = F.spectrum(om - shift, spec.eta, NSTEPS).cpu().numpy()
        bse.bse_status_read(plan)
        return float(np.sum(wgt * (e - target) ** 2)), e

    _, e0 = loss()
    assert np.abs(half - e0).max() / np.abs(e0).max() < 1e-5      # recursion converged at eta
    g = 2.0 * wgt * (e0 - target)
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_BACKWARD, NSTEPS) // 8 + 1, dtype=torch.complex64,
                     device="cuda")
    dd = torch.zeros(1, dtype=torch.float64, device="cuda")
    drx, drd = torch.zeros_like(F.rho_x), torch.zeros_like(F.rho_dir)
    dW, dH = torch.zeros_like(W), torch.zeros_like(F.H)
    bse.bse_spectrum_backward(plan, 0, F.H, F.P, NSTEPS, om, spec.eta, _dev(g, torch.float64), F.rho_x, F.rho_dir, W,
                              dd, dH, drx, drd, dW, ws)
    bse.bse_status_read(plan)
    fd = richardson_fd(lambda h: loss(shift=h)[0], 2e-5)
    assert abs(float(dd.item()) - fd) < 1e-4 * abs(fd), (float(dd.item()), fd)
    dWn = dW.cpu().numpy().astype(np.complex128)
    W0, dirs = w_directions(s)
    for name, D, h in dirs:
        an = float(np.sum(dWn.real * D.real + dWn.imag * D.imag))
        fdw = richardson_fd(lambda t: loss(_dev(W0 + t * D, torch.complex64))[0], h)
        assert abs(an - fdw) < 1e-4 * abs(fdw), (name, an, fdw, abs(an - fdw) / abs(fdw))
