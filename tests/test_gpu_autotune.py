"""Pair-kernel variants and their autotuner (through the C ABI).

The pruned-FFT variants only re-partition the same arithmetic (per z-line FFTs, per-slab y FFTs, the
x DFT accumulated slab by slab in the same order), so they must give bit-identical pair densities.
The plane-wave correlation variant (rows = 0, the default where it is compiled) sums the same
quantity in another order: it and every FFT variant are compared with the oracle (1e-5).
"""
import json

import numpy as np
import pytest

from oracle import pair as op
from synth import config_spec, generate, slab_batch_specs

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


def _cells():
    hexs = slab_batch_specs(0)
    out = [config_spec("fcc_8x8x8_3v4c").replace(name="fcc32_small", nk=(2, 2, 2), nsteps=10, nw=50)]
    for nv, nc in ((1, 1), (2, 2), (1, 3), (3, 3)):
        out.append(hexs[5].replace(name=f"hex_{nv}v{nc}c", nk=(6, 6, 1), nv=nv, nc=nc, nsteps=10, nw=50))
    return out


@pytest.mark.parametrize("spec", _cells(), ids=lambda s: s.name)
def test_variants_bit_identical_and_match_oracle(bse, spec):
    from paper_1206_3518_gb300.pipeline import Forward
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    variants, default = bse.bse_pair_variants(plan, 0)
    assert variants and default == variants[0]["index"]
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    coef, en = _dev(s.coef, torch.complex64), _dev(s.energies, torch.float64)
    assert any(v["rows"] == 0 for v in variants) and variants[0]["rows"] == 0    # correlation kernel first
    g = op.exchange_rho(spec, s.gk, s.coef)
    ref, cref, outs = None, None, []
    for v in variants:
        bse.bse_set_pair_variant(plan, 0, v["index"])
        assert bse.bse_pair_variants(plan, 0)[1] == v["index"]
        F.rho_x.zero_()
        F.rho_dir.zero_()
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None, 0,
                               0, F.ws_pair)
        q0, q1 = F.chunks[0]
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        bse.bse_status_read(plan)
        got = (F.rho_x.cpu().numpy(), F.rho_dir.cpu().numpy())
        outs.append(got)
        rx = got[0][:, :g.shape[1]]
        assert np.abs(rx - g).max() / np.abs(g).max() < 1e-5, v        # exchange densities vs the oracle
        if v["rows"] == 0:
            # the correlation kernels (plain and pipelined gather, direct set merged or split over two CTAs)
            # run the same sums in the same order
            if cref is None:
                cref = got
            else:
                assert np.array_equal(got[0], cref[0]) and np.array_equal(got[1], cref[1]), v
            continue
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), v
    bse.bse_set_pair_variant(plan, 0, -1)
    # direct densities: correlation and FFT variants agree to FP32 rounding
    dc, df = outs[0][1], ref[1]
    assert np.abs(dc - df).max() < 1e-5 * np.abs(df).max()
    with pytest.raises(bse.BseError):
        bse.bse_set_pair_variant(plan, 0, 10 ** 6)


def test_autotune_picks_fastest_and_caches(bse, tmp_path):
    from paper_1206_3518_gb300 import autotune
    from paper_1206_3518_gb300.pipeline import Forward
    spec = slab_batch_specs(0)[5].replace(name="tune", nk=(24, 24, 1), nv=1, nc=1)
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    variants, _ = bse.bse_pair_variants(plan, 0)
    assert len(variants) == 6            # the correlation kernel (three schedules) and three FFT tile shapes
    F = Forward(plan, 0, nsteps=10, nw=50, qchunk=32)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE, _dev(s.coef, torch.complex64),
                           _dev(s.energies, torch.float64), None, None, None, 0, 0, F.ws_pair)
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(plan, 0, F, reps=2, cache_path=cache)
    assert not r["cached"]
    ms = r["ms"]
    assert len(ms) == 6 and all(t > 0 for t in ms.values())
    assert r["variant"]["index"] == int(min(ms, key=ms.get))
    assert bse.bse_pair_variants(plan, 0)[1] == r["variant"]["index"]
    stored = json.load(open(cache))
    assert len(stored) == 1
    plan2 = bse.Plan([spec])
    r2 = autotune.tune(plan2, 0, F, cache_path=cache)
    assert r2["cached"] and r2["variant"]["index"] == r["variant"]["index"]
    assert bse.bse_pair_variants(plan2, 0)[1] == r["variant"]["index"]


def test_autotune_tensor_candidate(bse, tmp_path):
    """For a mixed-precision build the tensor-core route is one more timed candidate: the faster of it and
    the best variant is recorded on the Forward, which build() then follows, and the cache keeps it."""
    from paper_1206_3518_gb300 import autotune
    from paper_1206_3518_gb300.pipeline import Forward
    spec = slab_batch_specs(0)[5].replace(name="tune_tc", nk=(24, 24, 1), nv=1, nc=2)
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    assert plan.info(0)["tensor_pair"] == 1
    F = Forward(plan, 0, nsteps=10, nw=50, qchunk=48)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE, _dev(s.coef, torch.complex64),
                           _dev(s.energies, torch.float64), None, None, None, 0, 0, F.ws_pair)
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(plan, 0, F, reps=2, cache_path=cache, with_tensor=True)
    assert isinstance(r["tensor"], bool) and r["ms"]["tensor"] > 0
    best_variant = r["ms"][str(r["variant"]["index"])]
    assert r["tensor"] == (r["ms"]["tensor"] < best_variant)
    assert F.tensor_choice == r["tensor"]
    print(f"tensor route {r['ms']['tensor']:.3f} ms against variant {r['variant']['index']} {best_variant:.3f} ms: "
          f"{'tensor' if r['tensor'] else 'variant'}")
    F2 = Forward(plan, 0, nsteps=10, nw=50, qchunk=48)
    r2 = autotune.tune(plan, 0, F2, cache_path=cache, with_tensor=True)
    assert r2["cached"] and r2["tensor"] == r["tensor"] and F2.tensor_choice == r["tensor"]
