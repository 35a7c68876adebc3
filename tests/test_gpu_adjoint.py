"""Adjoint of the spectrum (step A9) through the C ABI, against the oracle and finite differences.

Loss L = sum_w weight(w) (eps_2(w) - target(w))^2.  The same dL/deps_2 (from the oracle's
dense spectrum) feeds both sides, so the comparison isolates the adjoint.  With nsteps = dim
the Krylov space is complete and the Krylov resolvent is exact.
"""
import numpy as np
import pytest

from oracle import adjoint as oa
from oracle import spectrum as osp

from gradcheck import richardson_fd, w_directions

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


@pytest.fixture(scope="module")
def setup(bse, cfg1, cfg1_oracle):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = cfg1.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.dim, nw=spec.nw, keep_rho_dir=True)
    W = _dev(cfg1.W, torch.complex64)
    en = _dev(cfg1.energies, torch.float64)
    F.build(_dev(cfg1.coef, torch.complex64), en, W, spec.delta)
    om = _dev(cfg1.omega, torch.float64)
    H, P = cfg1_oracle["H"], cfg1_oracle["P"]
    e2 = osp.eps2_dense(spec, H, P, cfg1.omega, spec.eta)
    target = 0.8 * e2 + 0.05 * e2.max() * np.sin(cfg1.omega / 0.05)
    weight = np.full(spec.nw, 1.0 / spec.nw)
    g = 2.0 * weight * (e2 - target)
    return dict(plan=plan, F=F, W=W, en=en, om=om, g=g, target=target, weight=weight)


def _backward(bse, S, spec, nsteps):
    F = S["F"]
    ws = torch.empty(bse.bse_workspace_size(S["plan"], 0, bse.BSE_WS_BACKWARD, nsteps) // 8 + 1,
                     dtype=torch.complex64, device="cuda")
    dd = torch.zeros(1, dtype=torch.float64, device="cuda")
    drx = torch.zeros_like(F.rho_x)
    drd = torch.zeros_like(F.rho_dir)
    dW = torch.zeros_like(S["W"])
    dH = torch.zeros_like(F.H)
    gdev = _dev(S["g"], torch.float64)
    bse.bse_spectrum_backward(S["plan"], 0, F.H, F.P, nsteps, S["om"], spec.eta, gdev, F.rho_x, F.rho_dir, S["W"],
                              dd, dH, drx, drd, dW, ws)
    bse.bse_status_read(S["plan"])
    return float(dd.item()), dH.cpu().numpy(), drx.cpu().numpy(), drd.cpu().numpy(), dW.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_adjoint_matches_oracle_dense_gradient(bse, setup, cfg1, cfg1_oracle):
    spec = cfg1.spec
    dd, dH, drx, drd, dW = _backward(bse, setup, spec, spec.dim)
    od, odrx, odfac, odW, _ = oa.gradients(spec, cfg1.energies, spec.delta, cfg1_oracle["rho_x"],
                                           cfg1_oracle["factors"], cfg1.W, cfg1_oracle["P"], cfg1.omega, spec.eta,
                                           setup["g"])
    assert abs(dd - od) < 1e-4 * abs(od)
    assert _rel(drx[:, :113], odrx) < 1e-4
    assert _rel(dW, odW) < 1e-4
    # direct pair densities: GPU layout -> per block
    plan = setup["plan"]
    nv, nc = spec.nv, spec.nc
    got = {}
    base = 0
    for iq in range(spec.nkpt):
        blk, _ = bse.bse_pair_blocks(plan, 0, iq)
        ng = len(bse.bse_gvectors(plan, 0, iq, 1))
        nb = len(blk)
        for t, (ik, ik2) in enumerate(blk):
            rv = drd[base + t * nv * nv: base + (t + 1) * nv * nv, :ng].reshape(nv, nv, ng)
            rc = drd[base + nb * nv * nv + t * nc * nc: base + nb * nv * nv + (t + 1) * nc * nc, :ng].reshape(nc, nc, ng)
            got[(int(ik), int(ik2))] = (rv, rc)
        base += nb * (nv * nv + nc * nc)
    scale = max(max(np.abs(a).max(), np.abs(b).max()) for a, b in odfac)
    worst = 0.0
    for (ik, ik2, _, _, _), (grv, grc) in zip(cfg1_oracle["factors"], odfac):
        a, b = got[(ik, ik2)]
        worst = max(worst, np.abs(a - grv).max(), np.abs(b - grc).max())
    assert worst / scale < 1e-4
    # dL/dH (Hermitian part) against the oracle's dense G
    G = oa.grad_h(spec, cfg1_oracle["H"], cfg1_oracle["P"], cfg1.omega, spec.eta, setup["g"])
    Gh = 0.5 * (G + G.conj().T)
    assert _rel(dH, Gh) < 1e-4


def _loss_gpu(bse, S, spec, nsteps, omega_shift=0.0, W=None):
    F = S["F"]
    if W is not None:
        F.build(_dev(S["coef"], torch.complex64), S["en"], W, spec.delta)
    om = S["om"] - omega_shift
    eps = F.spectrum(om, spec.eta, nsteps=nsteps).cpu().numpy()
    bse.bse_status_read(S["plan"])
    r = eps - S["target"]
    return float(np.sum(S["weight"] * r * r)), eps


def test_delta_gradient_matches_finite_difference_of_gpu_forward(bse, setup, cfg1):
    """Delta shifts H by Delta*I, i.e. eps_2(w; Delta + h) = eps_2(w - h; Delta): FD through the frequency grid."""
    spec = cfg1.spec
    n = spec.dim
    _, eps0 = _loss_gpu(bse, setup, spec, n)
    g = 2.0 * setup["weight"] * (eps0 - setup["target"])
    S = dict(setup, g=g)
    dd = _backward(bse, S, spec, n)[0]
    h = 2e-5
    fd = (_loss_gpu(bse, setup, spec, n, omega_shift=h)[0] - _loss_gpu(bse, setup, spec, n, omega_shift=-h)[0]) / (2 * h)
    assert abs(dd - fd) < 1e-4 * abs(fd)


def test_w_directional_derivatives_match_finite_differences_of_gpu_forward(bse, setup, cfg1):
    """dL/dt of L(W + t D) along two Hermitian, reciprocal directions D, against Richardson-combined
    central differences of the GPU forward (H rebuilt from W + t D each time).

    Each directional derivative sums the gradient over every entry of W, so the FP32 rounding of
    the rebuilt H (which limits a single-entry difference to ~1e-2) stays well below the signal;
    steps h and 2h with h = 4e-2 / max|D/W| (the h^2 term cancels; the FP32 rounding noise of the
    rebuilt H shrinks with 1/h, the h^4 term grows with the largest relative change of W).
    """
    spec = cfg1.spec
    n = spec.dim
    S = dict(setup, coef=cfg1.coef)
    try:
        _, eps0 = _loss_gpu(bse, S, spec, n, W=setup["W"])
        g = 2.0 * setup["weight"] * (eps0 - setup["target"])
        dW = _backward(bse, dict(setup, g=g), spec, n)[4].astype(np.complex128)
        W0, dirs = w_directions(cfg1)
        for name, D, h in dirs:
            an = float(np.sum(dW.real * D.real + dW.imag * D.imag))
            fd = richardson_fd(lambda t: _loss_gpu(bse, S, spec, n, W=_dev(W0 + t * D, torch.complex64))[0], h)
            assert abs(an - fd) < 1e-4 * abs(fd), (name, an, fd, abs(an - fd) / abs(fd))
    finally:
        _loss_gpu(bse, S, spec, n, W=setup["W"])


def test_autograd_function_matches_direct_adjoint(bse, setup, cfg1):
    from paper_1206_3518_gb300.autograd import eps2 as eps2_fn
    spec = cfg1.spec
    F = setup["F"]
    delta = torch.tensor(spec.delta, dtype=torch.float64, device="cuda", requires_grad=True)
    W = setup["W"].clone().requires_grad_(True)
    rx = F.rho_x.clone().requires_grad_(True)
    rd = F.rho_dir.clone().requires_grad_(True)
    e = eps2_fn(delta, W, rx, rd, setup["plan"], 0, setup["en"], F.P, setup["om"], spec.eta, spec.dim)
    w = torch.as_tensor(setup["weight"], device="cuda")
    t = torch.as_tensor(setup["target"], device="cuda")
    loss = torch.sum(w * (e - t) ** 2)
    loss.backward()
    g = (2.0 * w * (e.detach() - t)).cpu().numpy()
    dd, _, drx, drd, dW = _backward(bse, dict(setup, g=g), spec, spec.dim)
    assert abs(float(delta.grad) - dd) <= 1e-9 * abs(dd)
    assert np.array_equal(W.grad.cpu().numpy(), dW)
    assert np.array_equal(rx.grad.cpu().numpy(), drx)
    assert np.array_equal(rd.grad.cpu().numpy(), drd)
