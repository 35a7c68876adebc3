"""Failure detection on the GPU without a fault: a grid-barrier wait that runs out.

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
