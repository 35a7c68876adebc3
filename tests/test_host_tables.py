"""Host logic of the C ABI (no GPU): symbol exports, bit-exact A0 tables against the oracle."""
import re

import numpy as np
import pytest

from oracle import geometry as geo
from oracle import kernel as ok
from oracle import spectrum as osp
from synth import SystemSpec, config_spec, slab_batch_specs


@pytest.fixture(scope="module")
def bse():
    import __graft_entry__ as ge
    ge.build()
    from paper_1206_3518_gb300 import bse as b
    b.load()
    return b


def test_library_exports_every_declared_symbol(bse):
    import os
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "bse.h")).read()
    declared = set(re.findall(r"^(?:bse_status|const char\*)\s+(bse_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 14
    lib = bse.load()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(bse.EXPORTED)


@pytest.mark.parametrize("spec", [config_spec("fcc_4x4x4_3v3c"), slab_batch_specs(0)[1],
                                  SystemSpec("fcc_tiny", "fcc", 10.0, 0.0, (2, 2, 2), 2, 2, 1.0, (8, 8, 8), "3d")])
def test_spheres_bit_exact_against_oracle(bse, spec):
    plan = bse.Plan([spec], host_only=True)
    kr = geo.mesh_offsets(spec)
    step = max(1, spec.nkpt // 40)
    for ik in range(0, spec.nkpt, step):
        g = bse.bse_gvectors(plan, 0, ik, 0)
        assert np.array_equal(g, geo.sphere(spec, tuple(kr[ik])))
        assert np.array_equal(bse.bse_gvectors(plan, 0, ik, 1), g)


def test_blocks_and_folds_bit_exact_against_oracle(bse, cfg1):
    spec = cfg1.spec
    plan = bse.Plan([spec], host_only=True)
    kr = geo.mesh_offsets(spec)
    seen = set()
    for iq in range(spec.nkpt):
        blk, g0 = bse.bse_pair_blocks(plan, 0, iq)
        assert np.all(np.diff(blk[:, 0]) > 0)                     # ascending k within a q
        for (ik, ik2), g in zip(blk, g0):
            assert ik <= ik2
            q, _, og0 = geo.fold(spec, kr[ik], kr[ik2])
            assert q == iq and np.array_equal(og0, g)
            seen.add((int(ik), int(ik2)))
    assert seen == set(geo.upper_blocks(spec))


def test_info_constants_match_oracle(bse, cfg1):
    spec = cfg1.spec
    inf = bse.Plan([spec], host_only=True).info(0)
    assert inf["dim"] == 576 and inf["nblocks"] == 2080 and inf["ng0"] == 113
    assert inf["norm"] == ok.norm_factor(spec)
    assert abs(inf["prefactor"] - osp.prefactor(spec)) <= 1e-18
    assert bse.bse_rho_dir_count(bse.Plan([spec], host_only=True), 0, 0, 64) == 2080 * (9 + 9)


@pytest.mark.parametrize("bad, msg", [
    (dict(fft=(9, 9, 9)), "divide 192"),
    (dict(fft=(8, 8, 8)), "alias-free"),
    (dict(nk=(4, 4, 2)), "nk1 = nk2 = nk3"),
    (dict(nv=5), "nv, nc"),
])
def test_invalid_systems_rejected(bse, bad, msg):
    spec = config_spec("fcc_4x4x4_3v3c").replace(**bad)
    with pytest.raises(bse.BseError) as e:
        bse.Plan([spec], host_only=True)
    assert e.value.code == bse.BSE_ERR_ARG and msg in str(e.value)


def test_host_only_plan_refuses_compute(bse, cfg1):
    plan = bse.Plan([cfg1.spec], host_only=True)
    with pytest.raises(bse.BseError) as e:
        bse.load().bse_apply_H(plan.handle, 0, None, None, None, 1, None)
        bse._check(bse.load().bse_apply_H(plan.handle, 0, None, None, None, 1, None))
    assert e.value.code == bse.BSE_ERR_ARG


@pytest.mark.parametrize("name", ["fcc_4x4x4_3v3c", "fcc_8x8x8_3v4c", "hex6"])
def test_symmetry_tables_bit_exact_vs_oracle(name):
    """Point group order, irreducible q points, per-q maps and sphere permutations of the host planner
    against oracle/symmetry.py (integer work: bit-exact)."""
    from oracle import symmetry as sy
    from paper_1206_3518_gb300 import bse
    from synth import config_spec, slab_batch_specs
    spec = slab_batch_specs(0)[5].replace(name="hex6", nk=(6, 6, 1)) if name == "hex6" else config_spec(name)
    plan = bse.bse_plan_create_host([spec])
    nops, ibz, qmap, perm = bse.bse_symmetry(plan, 0)
    ops = sy.point_group(spec)
    oibz, oqmap = sy.reduce_mesh(spec, ops)
    assert nops == len(ops)
    assert ibz.tolist() == list(oibz)
    assert [tuple(r) for r in qmap.tolist()] == [tuple(m) for m in oqmap]
    for iq in range(spec.nkpt):
        p = sy.sphere_perm(spec, iq, oibz, oqmap, ops)
        assert perm[iq, :len(p)].tolist() == p.tolist() and np.all(perm[iq, len(p):] == -1)


def test_new_entry_points_validate_arguments(bse, cfg1):
    """Host-side checks of the coupled, Ritz and symmetry calls: NULL or out-of-range arguments and
    host-only plans return an error status without touching a device."""
    import ctypes
    lib = bse.load()
    plan = bse.Plan([cfg1.spec], host_only=True)
    h = plan.handle
    # compute calls refuse a host-only plan
    for code in (lib.bse_build_coupling(h, 0, bse.BSE_BC_INIT, None, None, 0, 0, None, 0, None, None, 0, None),
                 lib.bse_spectrum_coupled(h, 0, None, None, None, 10, None, 0, 0.01, None, None, None, None, 0, None),
                 lib.bse_unfold_w(h, 0, None, None, 0, 1, None)):
        assert code == bse.BSE_ERR_ARG
    # bse_ritz needs its pointers and 1 <= nsteps <= 4096, and a workspace of the stated size
    assert lib.bse_ritz(None, None, 10, None, None, None, 0, None) == bse.BSE_ERR_ARG
    dummy = ctypes.c_void_p(16)
    assert lib.bse_ritz(dummy, dummy, 0, dummy, dummy, dummy, 1 << 30, None) == bse.BSE_ERR_ARG
    assert lib.bse_ritz(dummy, dummy, 5000, dummy, dummy, dummy, 1 << 30, None) == bse.BSE_ERR_ARG
    assert lib.bse_ritz(dummy, dummy, 100, dummy, dummy, dummy, 8, None) == bse.BSE_ERR_WORKSPACE
    # workspace sizes: coupled spectrum grows with nsteps, Ritz is 6 nsteps^2 doubles
    assert bse.bse_workspace_size(plan, 0, bse.BSE_WS_RITZ, 100) == 6 * 100 * 100 * 8
    assert (bse.bse_workspace_size(plan, 0, bse.BSE_WS_COUPLED, 200) >
            bse.bse_workspace_size(plan, 0, bse.BSE_WS_COUPLED, 100) > 0)
    assert bse.bse_workspace_size(plan, 0, bse.BSE_WS_COUPLING, 0) >= 576 * 113 * 8
    with pytest.raises(bse.BseError):
        bse.bse_workspace_size(plan, 0, bse.BSE_WS_RITZ, 0)
    # coupling vector count: 2 Nv Nc per upper block of the range
    blocks = sum(len(bse.bse_pair_blocks(plan, 0, q)[0]) for q in range(3))
    assert bse.bse_rho_cpl_count(plan, 0, 0, 3) == 2 * 9 * blocks
    # the symmetry tables are available on a host-only plan
    nops, ibz, qmap, perm = bse.bse_symmetry(plan, 0)
    assert nops == 48 and len(ibz) == 8 and qmap.shape == (64, 6)


def test_bench_pair_work_counts_the_correlation_loop(bse, cfg1):
    """bench.py's algorithmic work of the correlation kernel: sum over the upper blocks of
    NG(q) |S(k')| (Nv^2 + Nc^2) complex multiply-adds, recounted from the oracle's spheres."""
    import importlib.util
    import os
    spec = cfg1.spec
    path = os.path.join(os.path.dirname(__file__), "..", "bench.py")
    sp = importlib.util.spec_from_file_location("bench_mod", path)
    bench = importlib.util.module_from_spec(sp)
    sp.loader.exec_module(bench)
    plan = bse.Plan([spec], host_only=True)
    pw = bench.pair_work(plan, spec, plan.info(0))
    assert pw["method"] == "correlation" and pw["variant"] in (64, 65, 66)
    kr = geo.mesh_offsets(spec)
    npw = [len(geo.sphere(spec, tuple(k))) for k in kr]
    cmac = 0
    for ik, ik2 in geo.upper_blocks(spec):
        iq, iqv, _ = geo.fold(spec, kr[ik], kr[ik2])
        cmac += len(geo.sphere(spec, tuple(iqv))) * npw[ik2]
    assert pw["cmac"] == cmac * (spec.nv ** 2 + spec.nc ** 2)


def test_kpoint_symmetry_representatives_match_oracle(bse):
    """With k-point symmetry the plan keeps exactly the oracle's representative upper blocks."""
    from oracle import symmetry as sym
    for name in ("fcc_4x4x4_3v3c", "fcc_8x8x8_3v4c"):
        spec = config_spec(name).replace(symmetric=True, w_offdiag=0.0)
        plan = bse.Plan([spec], host_only=True)
        inf = plan.info(0)
        reps, _ = sym.reduce_blocks(spec)
        blocks = geo.upper_blocks(spec)
        got = set()
        for q in range(spec.nkpt):
            b, _ = bse.bse_pair_blocks(plan, 0, q)
            got |= {(int(x), int(y)) for x, y in b}
        assert got == {blocks[r] for r in reps}
        assert inf["kpoint_symmetry"] == 1 and inf["nblocks"] == len(reps)
        assert inf["nblocks"] + inf["nfill"] == len(blocks)
