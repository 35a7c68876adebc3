"""Failure detection on the GPU without a fault: a grid-barrier wait that runs out, and input scans.

With the wait limit forced to 0 every barrier wait of the spectrum kernel gives up at once; the
kernel must record BSE_ERR_TIMEOUT in the plan's status word and return (no hang), and the
context must stay usable: with the default limit restored the same spectrum is reproduced
bit for bit.
"""
import numpy as np
import pytest

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


def test_barrier_timeout_reports_status_and_context_survives(bse):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = SystemSpec("fail", "fcc", 10.0, 0.0, (3, 3, 3), 2, 2, 1.0, (8, 8, 8), "3d", nsteps=24, nw=100)
    s = generate(spec)
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    dev = lambda x, t: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=t)  # noqa: E731
    F.build(dev(s.coef, torch.complex64), dev(s.energies, torch.float64), dev(s.W, torch.complex64), spec.delta)
    om = dev(s.omega, torch.float64)
    ref = F.spectrum(om, spec.eta).clone()
    bse.bse_status_read(plan)
    try:
        bse.bse_set_wait_limit(0)
        F.spectrum(om, spec.eta)
        with pytest.raises(bse.BseError) as err:
            bse.bse_status_read(plan)
        assert err.value.code == bse.BSE_ERR_TIMEOUT
    finally:
        bse.bse_set_wait_limit(2_000_000_000)
    bse.bse_status_read(plan)                 # the status word was cleared by the read above
    again = F.spectrum(om, spec.eta)
    bse.bse_status_read(plan)
    assert torch.equal(again, ref)


def test_nonfinite_inputs_report_status(bse):
    """A NaN or an infinity planted on the host in coef, energies, a W row of the call's q range, H or P makes
    the call's input scan set BSE_ERR_NONFINITE; a NaN in a W row outside the range is not the call's input.
    After each bad call the clean inputs reproduce the clean results bit for bit."""
    from paper_1206_3518_gb300.pipeline import Forward
    spec = SystemSpec("nan", "fcc", 10.0, 0.0, (3, 3, 3), 2, 2, 1.0, (8, 8, 8), "3d", nsteps=24, nw=100)
    s = generate(spec)
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw, qchunk=9)
    dev = lambda x, t: torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=t)  # noqa: E731
    coef, en, W = dev(s.coef, torch.complex64), dev(s.energies, torch.float64), dev(s.W, torch.complex64)
    om = dev(s.omega, torch.float64)
    F.build(coef, en, W, spec.delta)
    ref_h = F.H.clone()
    ref = F.spectrum(om, spec.eta).clone()
    bse.bse_status_read(plan)

    def expect_nonfinite(fn):
        fn()
        with pytest.raises(bse.BseError) as err:
            bse.bse_status_read(plan)
        assert err.value.code == bse.BSE_ERR_NONFINITE

    bad = coef.clone()
    bad[5, 1, 3] = complex(float("nan"), 0.0)
    expect_nonfinite(lambda: F.build(bad, en, W, spec.delta))
    bad = en.clone()
    bad[2, 0] = float("inf")
    expect_nonfinite(lambda: F.build(coef, bad, W, spec.delta))
    q0, q1 = F.chunks[1]
    bad = W.clone()
    bad[q0 + 1, 2, 4] = complex(0.0, float("-inf"))
    expect_nonfinite(lambda: bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, bad, None,
                                                  spec.delta, bse.BSE_PREC_FP32, F.H, F.ws_kernel))
    bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, 0, F.chunks[0][1], bad, None, spec.delta,
                         bse.BSE_PREC_FP32, F.H, F.ws_kernel)
    bse.bse_status_read(plan)                 # the bad row lies outside this call's q range
    F.build(coef, en, W, spec.delta)
    bse.bse_status_read(plan)
    assert torch.equal(F.H, ref_h)
    Hc = F.H.clone()
    F.H[7, 11] = complex(float("nan"), float("nan"))
    expect_nonfinite(lambda: F.spectrum(om, spec.eta))
    F.H.copy_(Hc)
    Pc = F.P.clone()
    F.P[3] = complex(float("inf"), 0.0)
    expect_nonfinite(lambda: F.spectrum(om, spec.eta))
    F.P.copy_(Pc)
    again = F.spectrum(om, spec.eta)
    bse.bse_status_read(plan)
    assert torch.equal(again, ref)
