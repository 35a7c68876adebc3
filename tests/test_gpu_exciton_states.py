"""Exciton states (Eq. bse_eig) on the GPU: all eigenpairs of the fcc 4x4x4 3v3c Hamiltonian (dim 576) from a
Lanczos tridiagonalisation of full Krylov dimension, against the oracle's dense diagonalisation."""
import numpy as np
import pytest
import scipy.linalg

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


def _dev(x, dtype):
    return torch.as_tensor(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _states(bse, plan, H, x0, n):
    dim = H.shape[0]
    theta = torch.empty(n, dtype=torch.float64, device="cuda")
    A = torch.empty(n, dim, dtype=torch.complex64, device="cuda")
    ab = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    done = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_STATES, n) // 8 + 1, dtype=torch.complex64,
                     device="cuda")
    bse.bse_exciton_states(plan, 0, H, _dev(x0, torch.complex128), n, theta, A, ab, done, ws)
    bse.bse_status_read(plan)
    return theta.cpu().numpy(), A.cpu().numpy().astype(np.complex128), int(done.item())


def test_all_eigenpairs_match_dense_diagonalisation(bse, cfg1, cfg1_oracle):
    from paper_1206_3518_gb300.pipeline import Forward
    spec = cfg1.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    F.build(_dev(cfg1.coef, torch.complex64), _dev(cfg1.energies, torch.float64), _dev(cfg1.W, torch.complex64),
            spec.delta)
    bse.bse_status_read(plan)
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(spec.dim) + 1j * rng.standard_normal(spec.dim)
    theta, A, done = _states(bse, plan, F.H, x0, spec.dim)
    assert done == spec.dim
    Href = cfg1_oracle["H"]
    E, V = scipy.linalg.eigh(Href)
    scale = np.abs(E).max()
    err_e = np.abs(theta - E).max() / scale
    Hg = F.H.cpu().numpy().astype(np.complex128)
    res = np.abs(A @ Hg.T - theta[:, None] * A).max() / np.abs(Hg).max()        # rows: H A_l = theta_l A_l
    orth = np.abs(A.conj() @ A.T - np.eye(spec.dim)).max()
    gap = np.minimum(np.diff(E, prepend=-np.inf), np.diff(E, append=np.inf))
    iso = gap > 1e-4 * scale
    ov = np.abs(np.sum(A.conj() * V.T, axis=1))                                   # |<A_l, A_l^ref>|
    P = cfg1_oracle["P"]
    wg = np.abs(A.conj() @ P) ** 2
    wref = np.abs(V.conj().T @ P) ** 2
    eps_g = osp.prefactor(spec) * (spec.eta / ((cfg1.omega[:, None] - theta[None, :]) ** 2 + spec.eta ** 2)) @ wg
    eps_ref = osp.eps2_dense(spec, Href, P, cfg1.omega, spec.eta)
    err_eps = np.abs(eps_g - eps_ref).max() / eps_ref.max()
    print(f"exciton states (dim {spec.dim}): eigenvalues {err_e:.2e} of max |E|, residual {res:.2e}, "
          f"orthonormality {orth:.2e}, min overlap of {int(iso.sum())} isolated states {ov[iso].min():.6f}, "
          f"eps_2 from the eigenpairs {err_eps:.2e}; dark states (weight < 1e-8 of max): "
          f"{int((wref < 1e-8 * wref.max()).sum())}")
    assert err_e < 1e-6
    assert res < 1e-5
    assert orth < 1e-4
    assert ov[iso].min() > 1.0 - 1e-4
    assert np.abs(wg.sum() - np.vdot(P, P).real) < 1e-5 * np.vdot(P, P).real
    assert err_eps < 1e-5


def test_ritz_pairs_of_a_shorter_recursion(bse, cfg1, cfg1_oracle):
    """n < dim: the extreme Ritz values converge to the extreme eigenvalues, and every Ritz pair satisfies
    H A = theta A + residual in the Krylov space (the residual of pair l is |b_n y_l(n - 1)|)."""
    from paper_1206_3518_gb300.pipeline import Forward
    spec = cfg1.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    F.build(_dev(cfg1.coef, torch.complex64), _dev(cfg1.energies, torch.float64), _dev(cfg1.W, torch.complex64),
            spec.delta)
    rng = np.random.default_rng(9)
    x0 = rng.standard_normal(spec.dim) + 1j * rng.standard_normal(spec.dim)
    n = 160
    theta, A, done = _states(bse, plan, F.H, x0, n)
    assert done == n
    E = scipy.linalg.eigvalsh(cfg1_oracle["H"])
    assert abs(theta[0] - E[0]) < 1e-6 * np.abs(E).max()
    assert abs(theta[-1] - E[-1]) < 1e-6 * np.abs(E).max()
    assert np.all(np.diff(theta) >= 0)
    assert np.abs(A.conj() @ A.T - np.eye(n)).max() < 1e-4
