"""Direct pair densities on the tensor cores (bse_pair_densities with BSE_PD_DIRECT | BSE_PD_TENSOR) against
the oracle's plane-wave correlation (Eq. pair_density), through the C ABI.

The route splits every operand x = hi + lo in BF16 and accumulates hi.hi + hi.lo + lo.hi in FP32, so
each product carries ~2^-16 relative error: densities within 2e-5 of the largest density (the G = 0
overlaps of the diagonal blocks are summed in FP64 and held to FP32 rounding).  The rows of a tile
are the union of several blocks' spheres and its K positions the union of a region's spheres, so
these tests also pin the bookkeeping: every density of every block at its sphere position, whatever
the q chunks.
"""
import numpy as np
import pytest

from oracle import pair as op
from synth import SystemSpec, config_spec, generate
from synth.systems import slab_batch_specs

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


def _direct(bse, plan, F, s, chunks, tensor):
    """rho_dir of every chunk as {(ik, ik2): (rv, rc)}."""
    spec = s.spec
    nv, nc = spec.nv, spec.nc
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE, _dev(s.coef, torch.complex64),
                           _dev(s.energies, torch.float64), None, None, None, 0, 0, F.ws_pair)
    flags = bse.BSE_PD_DIRECT | (bse.BSE_PD_TENSOR if tensor else 0)
    out = {}
    for q0, q1 in chunks:
        F.rho_dir.fill_(float("nan"))
        bse.bse_pair_densities(plan, 0, flags, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        bse.bse_status_read(plan)
        rd = F.rho_dir.cpu().numpy()
        base = 0
        for iq in range(q0, q1):
            blk, _ = bse.bse_pair_blocks(plan, 0, iq)
            ng = len(bse.bse_gvectors(plan, 0, iq, 1))
            nb = len(blk)
            for t, (ik, ik2) in enumerate(blk):
                rv = rd[base + t * nv * nv: base + (t + 1) * nv * nv, :ng].reshape(nv, nv, ng)
                rc = rd[base + nb * nv * nv + t * nc * nc: base + nb * nv * nv + (t + 1) * nc * nc, :ng]
                out[(int(ik), int(ik2))] = (rv.copy(), rc.reshape(nc, nc, ng).copy())
            base += nb * (nv * nv + nc * nc)
    return out


def _check_against_oracle(spec, s, got, pairs=None):
    keys = sorted(got) if pairs is None else pairs
    worst, scale, g0 = 0.0, 0.0, 0.0
    for ik, ik2 in keys:
        iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
        gv, gc = got[(ik, ik2)]
        assert np.isfinite(gv).all() and np.isfinite(gc).all(), (ik, ik2)
        worst = max(worst, np.abs(gv - rv).max(), np.abs(gc - rc).max())
        scale = max(scale, np.abs(rv).max(), np.abs(rc).max())
        if ik == ik2:           # G = 0 overlaps of the diagonal blocks (FP64 sums)
            g0 = max(g0, np.abs(gv[:, :, 0] - rv[:, :, 0]).max(), np.abs(gc[:, :, 0] - rc[:, :, 0]).max())
    return worst / scale, g0 / scale


@pytest.mark.parametrize("name,nchunks", [("fcc_4x4x4_3v3c", 1), ("fcc_4x4x4_3v3c", 3), ("side_3v2c", 2),
                                          ("hex_1v2c", 2)])
def test_every_block_matches_oracle(bse, name, nchunks):
    from paper_1206_3518_gb300.pipeline import Forward
    if name == "side_3v2c":
        spec = SystemSpec(name, "fcc", 10.0, 0.0, (3, 3, 3), 3, 2, 1.0, (8, 8, 8), "3d", nsteps=20, nw=150)
    elif name == "hex_1v2c":
        spec = slab_batch_specs(0)[5].replace(name=name, nk=(6, 6, 1), nv=1, nc=2, nsteps=20, nw=150)
    else:
        spec = config_spec(name)
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    inf = plan.info(0)
    assert inf["tensor_pair"] == 1
    nq = inf["nq"]
    edges = np.linspace(0, nq, nchunks + 1).astype(int)
    chunks = [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:])]
    F = Forward(plan, 0, nsteps=10, nw=10, qchunk=max(b - a for a, b in chunks))
    got = _direct(bse, plan, F, s, chunks, tensor=True)
    assert len(got) == inf["nblocks"]
    err, err0 = _check_against_oracle(spec, s, got)
    ref32 = _direct(bse, plan, F, s, chunks, tensor=False)
    d32 = max(max(np.abs(got[key][0] - ref32[key][0]).max(), np.abs(got[key][1] - ref32[key][1]).max())
              for key in got)
    scale32 = max(max(np.abs(v[0]).max(), np.abs(v[1]).max()) for v in ref32.values())
    print(f"{name} ({nchunks} chunks, region {inf['tc_region']}, K {inf['tc_kpad']}): tensor-core direct densities "
          f"vs the oracle {err:.2e} of the largest (diagonal G = 0 overlaps {err0:.2e}); vs the FP32 correlation "
          f"kernel {d32 / scale32:.2e}")
    assert err < 2e-5
    assert err0 < 1e-6
    assert d32 / scale32 < 2e-5


def test_chunking_does_not_change_the_densities(bse, cfg1):
    """A block's densities depend on its own rows and its region's K layout only: the same values for
    one q chunk and for three."""
    from paper_1206_3518_gb300.pipeline import Forward
    spec = cfg1.spec
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=10, nw=10, qchunk=64)
    a = _direct(bse, plan, F, cfg1, [(0, 64)], tensor=True)
    b = _direct(bse, plan, F, cfg1, [(0, 20), (20, 41), (41, 64)], tensor=True)
    diff = max(max(np.abs(a[k][0] - b[k][0]).max(), np.abs(a[k][1] - b[k][1]).max()) for k in a)
    same = all(np.array_equal(a[k][0], b[k][0]) and np.array_equal(a[k][1], b[k][1]) for k in a)
    print(f"one chunk vs three: max difference {diff:.2e} (bit-identical: {same})")
    assert diff < 1e-7


def test_fcc8_sampled_blocks_full_size(bse):
    """fcc 8x8x8 3v4c at full size (regions of the plan's shape): a seeded sample of 400 upper blocks of every
    chunk of the bench's launch configuration against the oracle."""
    from paper_1206_3518_gb300.pipeline import Forward
    spec = config_spec("fcc_8x8x8_3v4c")
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    F = Forward(plan, 0, nsteps=10, nw=10, qchunk=103)
    got = _direct(bse, plan, F, s, F.chunks, tensor=True)
    keys = sorted(got)
    rng = np.random.default_rng(3)
    pick = [keys[i] for i in rng.choice(len(keys), 400, replace=False)]
    pick += [(k, k) for k in range(0, spec.nkpt, 37)]
    err, err0 = _check_against_oracle(spec, s, got, pick)
    print(f"fcc_8x8x8_3v4c: {len(pick)} sampled blocks of {len(keys)}: tensor-core direct densities vs the oracle "
          f"{err:.2e} of the largest (diagonal G = 0 {err0:.2e})")
    assert err < 2e-5 and err0 < 1e-6


def test_tensor_flag_arguments(bse, cfg1):
    from paper_1206_3518_gb300.pipeline import Forward
    plan = bse.Plan([cfg1.spec])
    F = Forward(plan, 0, nsteps=10, nw=10)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE, _dev(cfg1.coef, torch.complex64), None, None, None, None,
                           0, 0, F.ws_pair)
    with pytest.raises(bse.BseError) as e:
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT | bse.BSE_PD_TENSOR, None, None, None, None, F.rho_dir, 3,
                               3, F.ws_pair)
    assert e.value.code == bse.BSE_ERR_ARG
