"""bse_spectrum_static: the spectrum entry point for callers that cannot allocate device memory.

Some callers run the spectrum where they cannot call cudaMalloc - for example behind a
foreign-function boundary where the host framework owns every device buffer and hands over
only inputs and outputs.  bse_spectrum_static takes its scratch from a fixed 48 MiB array
inside the library instead of a caller workspace.  This test checks, through the C ABI, that
two calls in a row give the same spectrum as bse_spectrum with a caller workspace, and that a
request larger than the array is refused before any GPU work.  It sits in a file of its own
that pytest collects last, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bse():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_1206_3518_gb300 import bse as b
    b.load()
    return b


def test_static_scratch_spectrum_matches_workspace_spectrum(bse):
    from paper_1206_3518_gb300.pipeline import Forward
    from synth import config_spec, generate

    s = generate(config_spec("fcc_4x4x4_3v3c"))
    spec = s.spec
    dev = torch.device("cuda")
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    F.build(torch.as_tensor(s.coef, dtype=torch.complex64, device=dev),
            torch.as_tensor(s.energies, device=dev),
            torch.as_tensor(s.W, dtype=torch.complex64, device=dev), spec.delta)
    om = torch.as_tensor(s.omega, device=dev)
    ref = F.spectrum(om, spec.eta).clone()
    ref_ab = F.ab.clone()
    bse.bse_status_read(plan)
    peak = float(ref.abs().max())
    for _ in range(2):                                  # two calls in a row share the scratch
        eps2 = torch.full((spec.nw,), float("nan"), dtype=torch.float64, device=dev)
        ab = torch.full((2 * spec.nsteps,), float("nan"), dtype=torch.float64, device=dev)
        done = torch.zeros(1, dtype=torch.int32, device=dev)
        bse.bse_spectrum_static(plan, 0, F.H, F.P, spec.nsteps, om, spec.eta, eps2, ab, done)
        bse.bse_status_read(plan)
        assert int(done.item()) == spec.nsteps
        assert float((eps2 - ref).abs().max()) < 1e-5 * peak
        assert float((ab - ref_ab).abs().max()) < 1e-5 * float(ref_ab.abs().max())


def test_static_scratch_rejects_requests_beyond_its_size(bse):
    from synth import config_spec

    spec = config_spec("fcc_8x8x8_3v4c")                # dim 6144: 3000 steps need ~300 MB of scratch
    plan = bse.Plan([spec])
    dev = torch.device("cuda")
    small = torch.zeros(4, dtype=torch.complex128, device=dev)
    om = torch.zeros(4, dtype=torch.float64, device=dev)
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    done = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(bse.BseError) as e:
        bse.bse_spectrum_static(plan, 0, small, small, 3000, om, 0.01, out, out, done)
    assert e.value.code == bse.BSE_ERR_ARG and "exceeds" in str(e.value)
