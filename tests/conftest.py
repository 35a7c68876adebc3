import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session")
def tiny_spec():
    """A few-G FCC cell small enough for brute-force real-space sums (alias-free 8^3 grid)."""
    from synth import SystemSpec
    return SystemSpec("fcc_tiny", "fcc", 10.0, 0.0, (2, 2, 2), 2, 2, 1.0, (8, 8, 8), "3d",
                      eps_inf=11.0, nsteps=16, nw=200)


@pytest.fixture(scope="session")
def cfg1():
    from synth import config_spec, generate
    return generate(config_spec("fcc_4x4x4_3v3c"))


@pytest.fixture(scope="session")
def cfg1_oracle(cfg1):
    """Oracle products for the 4x4x4 fcc system: rho_x, upper-block factors, H, P."""
    from oracle import kernel as ok, pair as op
    spec = cfg1.spec
    rho_x = op.exchange_rho(spec, cfg1.gk, cfg1.coef)
    factors = ok.direct_factors(spec, cfg1.gk, cfg1.coef)
    H = ok.hamiltonian_from_factors(spec, cfg1.energies, spec.delta, rho_x, factors, cfg1.W)
    P = op.dipole(spec, cfg1.gk, cfg1.coef, cfg1.energies)
    return {"rho_x": rho_x, "factors": factors, "H": H, "P": P}
