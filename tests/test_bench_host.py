"""Host-side pieces of bench.py that need no GPU: the oracle leg of the CPU baseline (its parity figures are
zero when the 'GPU' H is the oracle's own), the q-chunk sizing and the per-stage roofline arithmetic."""
import importlib.util
import os

import numpy as np
import pytest

from oracle import kernel as ok
from oracle import pair as op
from oracle import spectrum as osp
from synth import SystemSpec, config_spec, generate


def _bench():
    path = os.path.join(os.path.dirname(__file__), "..", "bench.py")
    sp = importlib.util.spec_from_file_location("bench_mod", path)
    mod = importlib.util.module_from_spec(sp)
    sp.loader.exec_module(mod)
    return mod


def test_cpu_baseline_parity_is_zero_on_the_oracle_h():
    spec = SystemSpec("bench_tiny", "fcc", 10.0, 0.0, (2, 2, 2), 2, 2, 2.0, (12, 12, 12), "3d", nsteps=12, nw=300)
    s = generate(spec)
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    H = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    eps = osp.eps2_haydock(spec, H, P, s.omega, spec.eta, spec.nsteps)[0]
    bench = _bench()
    out = bench.cpu_baseline(spec, s, H, H, eps, eps, spec.nsteps, budget_s=2.0)
    par = out["parity"]
    assert par["blocks"] >= 1
    assert par["kernel_rel_err_fp32"]["max"] < 1e-12
    assert par["eps2_rel_err_fp32_vs_oracle_haydock"] < 1e-12
    assert out["value"] > 0 and out["kind"] == "oracle"


def test_auto_qchunk_fits_the_budget():
    bse = pytest.importorskip("paper_1206_3518_gb300.bse")
    try:
        bse.load()
    except RuntimeError:
        pytest.skip("library not built")
    bench = _bench()
    spec = config_spec("fcc_8x8x8_3v4c")
    plan = bse.Plan([spec], host_only=True)
    nq = plan.info(0)["nq"]
    budget = 6e9
    ch = bench.auto_qchunk(plan, nq, budget)
    chunks = [(q, min(q + ch, nq)) for q in range(0, nq, ch)]
    rho = max(bse.bse_rho_dir_count(plan, 0, a, b) for a, b in chunks) * plan.info(0)["ng_max"] * 8
    assert rho + bse.bse_workspace_size(plan, 0, bse.BSE_WS_KERNEL, ch) <= budget
    if ch > 1:
        ch2 = -(-nq // (-(-nq // ch) - 1))
        chunks2 = [(q, min(q + ch2, nq)) for q in range(0, nq, ch2)]
        rho2 = max(bse.bse_rho_dir_count(plan, 0, a, b) for a, b in chunks2) * plan.info(0)["ng_max"] * 8
        assert rho2 + bse.bse_workspace_size(plan, 0, bse.BSE_WS_KERNEL, ch2) > budget


def test_auto_qchunk_whole_planes():
    """With align = a plane of the q mesh, chunks are whole planes (so every region of k' is full for each k)
    whenever one plane fits the budget, and still fit it; a budget that holds one plane only gives one plane;
    below that the chunks are smaller than a plane and fit."""
    bse = pytest.importorskip("paper_1206_3518_gb300.bse")
    try:
        bse.load()
    except RuntimeError:
        pytest.skip("library not built")
    bench = _bench()
    spec = config_spec("fcc_8x8x8_3v4c")
    plan = bse.Plan([spec], host_only=True)
    nq = plan.info(0)["nq"]
    plane = spec.nk[1] * spec.nk[2]

    def need(ch):
        chunks = [(q, min(q + ch, nq)) for q in range(0, nq, ch)]
        rho = max(bse.bse_rho_dir_count(plan, 0, a, b) for a, b in chunks) * plan.info(0)["ng_max"] * 8
        return rho + bse.bse_workspace_size(plan, 0, bse.BSE_WS_KERNEL, ch)

    one = need(plane)
    for budget in (6e9, 2.5 * one, one):
        ch = bench.auto_qchunk(plan, nq, budget, plane)
        assert ch % plane == 0 and need(ch) <= budget
    assert bench.auto_qchunk(plan, nq, one, plane) == plane
    ch = bench.auto_qchunk(plan, nq, 0.7 * one, plane)
    assert ch < plane and need(ch) <= 0.7 * one


def test_stage_rooflines_arithmetic():
    bench = _bench()
    spec = config_spec("fcc_12x12x12_4v4c")
    inf = {"dim": spec.dim, "nblocks": spec.nkpt * (spec.nkpt + 1) // 2, "ng_max": 531, "ng0": 531}
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1600.0, "sm_max_mhz": 2000.0}
    st = {n: 100.0 for n in bench.STAGES}
    pw = {"method": "correlation", "cmac": 1.0e12}
    r = bench.stage_rooflines(st, spec, inf, peaks, "measured", 8, pw, 1)
    assert abs(r["pair_direct"]["achieved"] - 8.0e12 / 0.1 / 1e12) < 1e-9
    assert abs(r["spectrum"]["achieved"] - spec.nsteps * 8.0 * spec.dim ** 2 / 0.1 / 1e9) < 1e-6
    assert r["direct_contract"]["bound"] == "tensor" and r["direct_contract"]["peak"] == 1600.0
    assert abs(r["pair_direct"]["peak"] - 152 * 128 * 2 * 2000.0 * 1e6 / 1e12) < 1e-9
