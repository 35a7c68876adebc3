"""Static RPA screening (bse_screening) and the (k, k+q) pair densities behind it, against the oracle."""
import numpy as np
import pytest

from oracle import pair as op
from oracle import screening as scr
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


def _run(bse, s, iterations=16, keep_rho=True):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = s.spec
    plan = bse.Plan([spec])
    inf = plan.info(0)
    nq, ng, dim = inf["nq"], inf["ng_max"], inf["dim"]
    F = Forward(plan, 0, nsteps=4, nw=8)
    coef, en = _dev(s.coef, torch.complex64), _dev(s.energies, torch.float64)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None, 0, 0,
                           F.ws_pair)
    rho = torch.zeros(nq * dim, ng, dtype=torch.complex64, device="cuda")
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_CHI0, None, None, None, None, rho, 0, nq, F.ws_pair)
    bse.bse_status_read(plan)
    rho_host = rho.cpu().numpy().copy().reshape(nq, dim, ng) if keep_rho else None
    W = torch.zeros(nq, ng, ng, dtype=torch.complex64, device="cuda")
    res = torch.zeros(nq, dtype=torch.float32, device="cuda")
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_SCREEN, nq) // 8, dtype=torch.complex64, device="cuda")
    bse.bse_screening(plan, 0, rho, en, F.P, 0, nq, iterations, W, res, ws)
    bse.bse_status_read(plan)
    return plan, rho_host, W.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("which", ["tiny", "fcc_4x4x4_3v3c"])
def test_screening_matches_oracle(bse, tiny_spec, which):
    spec = tiny_spec if which == "tiny" else config_spec(which)
    s = generate(spec)
    plan, rho, W, res = _run(bse, s)
    assert res.max() < 1e-5                                  # Newton-Schulz converged (FP32)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    qs = range(spec.nkpt) if which == "tiny" else (0, 1, 5, 21, 42, 63)
    for iq in qs:
        gq, rref, _ = scr.chi0_pair(spec, s, iq)
        ng = len(gq)
        got = rho[iq][:, :ng]
        assert np.abs(got - rref).max() < 1e-5 * np.abs(rref).max()
        wref = scr.screened_w(spec, s, iq, P)
        wg = W[iq][:ng, :ng]
        assert np.abs(wg - wref).max() < 1e-5 * np.abs(wref).max(), iq
        assert np.all(W[iq][ng:, :] == 0) and np.all(W[iq][:, ng:] == 0)


def test_screening_fcc8_full_size_sampled(bse):
    """fcc 8x8x8 3v4c (512 q, ng 314, K = 6144): W of q = 0 and two other q against the oracle."""
    spec = config_spec("fcc_8x8x8_3v4c")
    s = generate(spec, wdtype=np.complex64)
    plan, _, W, res = _run(bse, s, keep_rho=False)
    assert res.max() < 1e-5
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    for iq in (0, 77, 300):
        wref = scr.screened_w(spec, s, iq, P)
        ng = wref.shape[0]
        assert np.abs(W[iq][:ng, :ng] - wref).max() < 1e-5 * np.abs(wref).max(), iq
