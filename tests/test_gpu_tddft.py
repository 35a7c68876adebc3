"""Macroscopic dielectric function from TDDFT with local fields on the GPU (Sec. II A-B) against the oracle:
the symmetrised Adler-Wiser response chi~0(w), the ALDA kernel F and eps_M(w) = 1/[eps^-1]_00 for the RPA
and ALDA Dyson equations, through the C ABI."""
import numpy as np
import pytest

from oracle import pair as op
from oracle import tddft as td
from synth import SystemSpec, config_spec, generate

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


def _cases():
    return [SystemSpec("td_small", "fcc", 10.0, 0.0, (2, 2, 2), 2, 2, 2.0, (24, 24, 24), "3d", nsteps=20, nw=60),
            config_spec("fcc_4x4x4_3v3c")]


@pytest.mark.parametrize("spec", _cases(), ids=lambda s: s.name)
def test_optical_response_matches_oracle(bse, spec):
    from paper_1206_3518_gb300.pipeline import Forward
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    inf = plan.info(0)
    F = Forward(plan, 0, nsteps=10, nw=10)
    coef, en = _dev(s.coef, torch.complex64), _dev(s.energies, torch.float64)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None, 0, 0,
                           F.ws_pair)
    om = np.linspace(0.0, 0.8, 61)
    eta = 0.005
    ng = inf["ng0"]
    omega = _dev(om, torch.float64)
    chi = torch.empty(len(om), ng, ng, dtype=torch.complex64, device="cuda")
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_CHI0) // 8 + 1, dtype=torch.complex64, device="cuda")
    bse.bse_chi0_optical(plan, 0, F.rho_x, F.P, en, spec.delta, omega, eta, chi, ws)
    Fx = torch.empty(ng, ng, dtype=torch.complex64, device="cuda")
    wsa = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_ALDA) // 8 + 1, dtype=torch.complex64, device="cuda")
    bse.bse_xc_kernel_alda(plan, 0, F.ws_pair, Fx, wsa)
    wse = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_EPSM, len(om)) // 8 + 1, dtype=torch.complex64,
                      device="cuda")
    e_rpa = torch.empty(len(om), dtype=torch.complex128, device="cuda")
    e_alda = torch.empty(len(om), dtype=torch.complex128, device="cuda")
    bse.bse_epsilon_macro(plan, 0, chi, None, e_rpa, wse)
    bse.bse_epsilon_macro(plan, 0, chi, Fx, e_alda, wse)
    bse.bse_status_read(plan)

    P = op.dipole(spec, s.gk, s.coef, s.energies)
    ref_chi = td.chi0_bar(spec, s, om, eta, spec.delta, P)
    got_chi = chi.cpu().numpy()
    err_chi = np.abs(got_chi - ref_chi).max() / np.abs(ref_chi).max()
    ref_F = td.fxc_matrix(spec, s)
    err_F = np.abs(Fx.cpu().numpy() - ref_F).max() / np.abs(ref_F).max()
    ref_rpa = td.epsilon_macro(ref_chi)
    ref_alda = td.epsilon_macro(ref_chi, ref_F)
    err_rpa = np.abs(e_rpa.cpu().numpy() - ref_rpa).max() / np.abs(ref_rpa).max()
    err_alda = np.abs(e_alda.cpu().numpy() - ref_alda).max() / np.abs(ref_alda).max()
    print(f"{spec.name}: chi~0 {err_chi:.2e}, F {err_F:.2e}, eps_M RPA {err_rpa:.2e}, ALDA {err_alda:.2e} "
          f"(relative to the largest entry)")
    assert err_chi < 1e-5
    assert err_F < 1e-5
    assert err_rpa < 1e-4 and err_alda < 1e-4
    # local fields and the xc kernel change the answer well above the tolerance
    nlf = 1.0 - ref_chi[:, 0, 0]
    assert np.abs(ref_rpa - nlf).max() > 1e-3 * np.abs(ref_rpa).max()
    assert np.abs(ref_alda - ref_rpa).max() > 1e-4 * np.abs(ref_rpa).max()


def test_optical_response_arguments(bse):
    spec = _cases()[0]
    plan = bse.Plan([spec])
    inf = plan.info(0)
    ng = inf["ng0"]
    chi = torch.empty(3, ng, ng, dtype=torch.complex64, device="cuda")
    eps = torch.empty(3, dtype=torch.complex128, device="cuda")
    small = torch.empty(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(bse.BseError) as e:
        bse.bse_epsilon_macro(plan, 0, chi, None, eps, small)
    assert e.value.code == bse.BSE_ERR_WORKSPACE
