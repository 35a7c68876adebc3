"""Benchmark of the BSE hot path: one step = pair densities + Hamiltonian + Haydock spectrum.

Workload: fcc 8x8x8 k mesh, 3 valence + 4 conduction bands (dim 6144), ~301 plane
waves per sphere, 32^3 grid, 300 Haydock steps, 2000 frequencies, eta 0.05 eV
(synthetic inputs of the paper's bulk BSE shape).  Every input (u store 0.94 GB,
H 302 MB, W 404 MB) is larger than the 129 MB L2, so no flush is needed between
steps.  Multi-GPU runs are independent replicas (weak scaling); see the design doc.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a bounded
sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BSE kernel elements/s (dim^2 per full step: pair densities + H + Haydock eps_2)"
UNIT = "elements/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            idx = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", idx], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(x, world, device="cpu"):
    """The largest x over the ranks of the default process group (x itself for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_systems(dims, rank, world):
    """Indices of the systems rank owns: largest dim^2 first, each to the least-loaded rank (ties: lower
    rank).  Every rank computes the same assignment; no exchange is needed."""
    load = [0.0] * world
    owner = [0] * len(dims)
    for i in sorted(range(len(dims)), key=lambda i: (-dims[i] * dims[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[i] = r
        load[r] += float(dims[i]) * dims[i]
    return [i for i in range(len(dims)) if owner[i] == rank]


def workload_config(spec, ng_max):
    """The workload description shared by both arms of the bench."""
    return {"workload": f"{spec.name}: fcc a=10 bohr, {spec.nk[0]}x{spec.nk[1]}x{spec.nk[2]} k, "
                        f"{spec.nv}v{spec.nc}c, dim {spec.dim}, Ecut {spec.ecut} Ha (ng_max {ng_max}), grid "
                        f"{spec.fft[0]}x{spec.fft[1]}x{spec.fft[2]}, {spec.nsteps} Haydock steps, {spec.nw} w",
            "dim": spec.dim, "nblocks": spec.nkpt * (spec.nkpt + 1) // 2,
            "l2": "inputs larger than L2 (u 0.94 GB, H 0.30 GB, W 0.40 GB); no flush"}


def make_inputs(name):
    from synth import config_spec, generate
    import numpy as np
    spec = config_spec(name)
    s = generate(spec, wdtype=np.complex64)
    return spec, s


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    from paper_1206_3518_gb300 import bse
    from paper_1206_3518_gb300.pipeline import Forward

    spec, s = make_inputs(args.config)
    plan = bse.Plan([spec])
    inf = plan.info(0)
    dim = inf["dim"]
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
    coef_h = torch.as_tensor(s.coef.astype(np.complex64)).pin_memory()
    en_h = torch.as_tensor(s.energies).pin_memory()
    W_h = torch.as_tensor(s.W).pin_memory()
    om_h = torch.as_tensor(s.omega).pin_memory()
    coef, en, W, om = (coef_h.to(dev), en_h.to(dev), W_h.to(dev), om_h.to(dev))
    stream = torch.cuda.current_stream()
    prec = bse.BSE_PREC_BF16X3 if args.prec == "bf16x3" else bse.BSE_PREC_FP32

    ev_names = ["realspace+exchange", "init", "pair_direct", "direct_contract", "spectrum"]

    def step(record=None, w_ready=None, w_free=None):
        """w_ready: event after which W holds this step's screening (waited before the direct term);
        w_free: recorded once the direct term no longer reads W (the next upload may start)."""
        def mark(i):
            if record is not None:
                record[i].record(stream)
        mark(0)
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None,
                               0, 0, F.ws_pair)
        mark(1)
        bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, en, spec.delta, prec, F.H, None)
        mark(2)
        for q0, q1 in F.chunks:
            bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
            mark(3)
            if w_ready is not None:
                stream.wait_event(w_ready)
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, W, None, spec.delta, prec,
                                 F.H, F.ws_kernel)
            mark(4)
        if w_free is not None:
            w_free.record(stream)
        bse.bse_spectrum(plan, 0, F.H, F.P, spec.nsteps, om, spec.eta, F.eps2, F.ab, F.steps_done, F.ws_spec)
        mark(5)

    launches_per_step = 3 + 1 + 3 * len(F.chunks) + 1    # realspace, pair x, dipole, init, (pair d, gemm, block)*, haydock
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)

    clocks = Clocks()
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    stage_ms = {n: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs) for i, n in enumerate(ev_names)}
    bse.bse_status_read(plan)
    ms = max_over_ranks(ms, world, dev)
    ms_per_step = ms / args.steps

    # end to end through host buffers: inputs H2D from pinned memory, eps_2 D2H, every step.  The screening
    # W (the largest input) is uploaded on a second stream while the pair densities are computed.
    eps_host = torch.empty(spec.nw, dtype=torch.float64).pin_memory()
    h2d = coef_h.numel() * 8 + en_h.numel() * 8 + W_h.numel() * 8 + om_h.numel() * 8
    d2h = spec.nw * 8
    e_steps = max(1, min(args.steps, 3))
    side = torch.cuda.Stream()
    w_free = torch.cuda.Event()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    w_free.record(stream)
    for _ in range(e_steps):
        coef.copy_(coef_h, non_blocking=True)
        en.copy_(en_h, non_blocking=True)
        om.copy_(om_h, non_blocking=True)
        side.wait_event(w_free)
        with torch.cuda.stream(side):
            W.copy_(W_h, non_blocking=True)
        w_ready = torch.cuda.Event()
        w_ready.record(side)
        step(w_ready=w_ready, w_free=w_free)
        eps_host.copy_(F.eps2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e_steps

    # mixed precision: the same step with the BF16 hi/lo tensor-core contractions
    mixed = None
    if not args.no_mixed:
        eps_fp32 = F.eps2.clone()
        evm = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
        prec_save = prec
        prec = bse.BSE_PREC_BF16X3

        def step_mixed(record=None):
            def mark(i):
                if record is not None:
                    record[i].record(stream)
            mark(0)
            bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None,
                                   0, 0, F.ws_pair)
            mark(1)
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, en, spec.delta, prec, F.H, None)
            mark(2)
            for q0, q1 in F.chunks:
                bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1,
                                       F.ws_pair)
                mark(3)
                bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, W, None, spec.delta, prec,
                                     F.H, F.ws_kernel)
                mark(4)
            bse.bse_spectrum(plan, 0, F.H, F.P, spec.nsteps, om, spec.eta, F.eps2, F.ab, F.steps_done, F.ws_spec)
            mark(5)

        for _ in range(args.warmup):
            step_mixed()
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record(stream)
        for k in range(args.steps):
            step_mixed(evm[k])
        m1.record(stream)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        prec = prec_save
        ms_mixed = m0.elapsed_time(m1) / args.steps
        st_mixed = {n: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evm) for i, n in enumerate(ev_names)}
        err = float((F.eps2 - eps_fp32).abs().max() / eps_fp32.abs().max())
        w_side = min(spec.nv ** 2, spec.nc ** 2)
        ng = inf["ng_max"]
        issued = 24.0 * inf["nblocks"] * w_side * ng * ng / len(F.chunks)     # 3 splits x 8 flops per complex MAC
        mixed = {"prec": "bf16x3", "ms_per_step": ms_mixed, "value": world * dim * dim / (ms_mixed / 1e3),
                 "stages_ms": st_mixed, "eps2_rel_err_vs_fp32": err,
                 "direct_contract_speedup_vs_fp32": stage_ms["direct_contract"] / st_mixed["direct_contract"],
                 "direct_contract_issued_bf16_tflops_upper_bound": issued / (st_mixed["direct_contract"] / 1e3) / 1e12}
        step()       # restore the FP32 state
        torch.cuda.synchronize()

    screening = None
    if not args.no_screening and world == 1:
        screening = run_screening(args, dev, spec, s, coef, en, F)
        step()       # restore the step's own state
        torch.cuda.synchronize()

    # q-point symmetry (Sec. III A): W of the irreducible points only, unfolded on the device
    nops, ibz_q, _, _ = bse.bse_symmetry(plan, 0)
    W_ibz = W[torch.as_tensor(ibz_q.astype(np.int64), device=dev)].contiguous()
    W_full = torch.empty_like(W)
    bse.bse_unfold_w(plan, 0, W_ibz, W_full, 0, inf["nq"])
    torch.cuda.synchronize()
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    bse.bse_unfold_w(plan, 0, W_ibz, W_full, 0, inf["nq"])
    u1.record(stream)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    symmetry = {"ops": nops, "irreducible_q": int(len(ibz_q)), "q": inf["nq"],
                "w_bytes_irreducible": W_ibz.numel() * 8, "w_bytes_full": W.numel() * 8,
                "unfold_ms": u0.elapsed_time(u1)}
    del W_ibz, W_full

    peaks, src = _peaks()
    coupled = None
    if not args.no_coupled and world == 1:
        coupled = run_coupled(args, dev, spec, W, om, F, peaks)

    batch = None
    if not args.no_batch:
        batch = run_batch(args, dev, rank, world)

    # dominant stage: by measured time
    dom = max(stage_ms, key=stage_ms.get)
    roof = roofline(dom, stage_ms[dom], spec, inf, peaks, src, len(F.chunks), pair_work(plan, spec, inf))
    out = {
        "metric": METRIC, "value": world * dim * dim / (ms_per_step / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(spec, inf["ng_max"]),
                       precision=("complex64 (f32) contractions" if prec == 0 else "bf16x3 contractions") +
                       ", f64 Lanczos coefficients and continued fraction",
                       parallelism=f"replicas x{world}"),
        "stages_ms": stage_ms,
        "kernel_elements_per_s": dim * dim / ((ms_per_step - stage_ms["spectrum"]) / 1e3),
        "spectra_per_s": 1e3 / stage_ms["spectrum"],
        "roofline": roof, "clocks": ck,
        "e2e": {"value": world * dim * dim / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "mixed": mixed,
        "batch": batch,
        "screening": screening,
        "coupled": coupled,
        "symmetry": symmetry,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(spec, s, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_batch(args, dev, rank=0, world=1):
    """Layered 2D batch: 16 hexagonal sheets (dims 576..20736), BF16x3 contractions, autotuned pair tiles,
    per-system builds plus one batched persistent spectrum launch, the whole sequence replayed as one
    CUDA graph.  With several ranks the sheets are sharded (balanced by dim^2, no exchange) and the time
    is the slowest rank's.  Returns the summary for the JSON line."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1206_3518_gb300 import autotune, bse
    from paper_1206_3518_gb300.pipeline import Batch
    from synth import generate, slab_batch_specs

    all_specs = slab_batch_specs(0)
    mine = shard_systems([sp.dim for sp in all_specs], rank, world)
    specs = [all_specs[i] for i in mine]
    systems = [generate(sp, wdtype=np.complex64) for sp in specs]
    plan = bse.Plan(specs)
    nsteps, nw = specs[0].nsteps, specs[0].nw
    B = Batch(plan, nsteps, nw, qchunk=64)
    coefs = [torch.as_tensor(x.coef.astype(np.complex64)).to(dev) for x in systems]
    ens = [torch.as_tensor(x.energies).to(dev) for x in systems]
    Ws = [torch.as_tensor(x.W).to(dev) for x in systems]
    deltas = [sp.delta for sp in specs]
    om = torch.as_tensor(systems[0].omega).to(dev)
    eta = specs[0].eta
    tuned = []
    for i, F in enumerate(B.sys):
        bse.bse_pair_densities(plan, i, bse.BSE_PD_REALSPACE, coefs[i], ens[i], None, None, None, 0, 0, F.ws_pair)
        r = autotune.tune(plan, i, F)
        tuned.append(r["variant"]["index"])
    prec = bse.BSE_PREC_BF16X3

    def seq():
        B.build(coefs, ens, Ws, deltas, prec)
        B.spectrum(om, eta)

    seq()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        seq()
    for _ in range(max(1, args.warmup - 1)):
        g.replay()
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 3))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(reps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    bse.bse_status_read(plan)
    ms = max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)
    dims = [sp.dim for sp in all_specs]
    return {"workload": "16 hexagonal sheets (a 4.7, c 30 bohr, slab Coulomb), k meshes 24x24..48x48, 1-3 v and c "
                        "bands, 300 steps, 2000 w; BF16x3 contractions; one CUDA graph per batch and rank",
            "systems": len(all_specs), "dims": dims, "ms_per_batch": ms,
            "spectra_per_s": len(all_specs) / (ms / 1e3),
            "elements_per_s": float(sum(d * d for d in dims)) / (ms / 1e3),
            "pair_variants_rank0": tuned, "ranks": world, "scaling": "strong" if world > 1 else None,
            "graph_replays_timed": reps}


def run_screening(args, dev, spec, s, coef, en, F):
    """Static RPA screening of the bench workload (all q): (k, k+q) pair densities, eps, Newton-Schulz
    inverse, W.  Returns the summary for the JSON line (times by CUDA events)."""
    import torch
    from paper_1206_3518_gb300 import bse

    plan = F.plan
    inf = plan.info(0)
    nq, ng, dim = inf["nq"], inf["ng_max"], inf["dim"]
    iters = 16
    rho = torch.empty(nq * dim, ng, dtype=torch.complex64, device=dev)
    W = torch.empty(nq, ng, ng, dtype=torch.complex64, device=dev)
    res = torch.empty(nq, dtype=torch.float32, device=dev)
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_SCREEN, nq) // 8, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream()

    def once(ev=None):
        if ev:
            ev[0].record(stream)
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_CHI0, None, None, None, None, rho, 0, nq, F.ws_pair)
        if ev:
            ev[1].record(stream)
        bse.bse_screening(plan, 0, rho, en, F.P, 0, nq, iters, W, res, ws)
        if ev:
            ev[2].record(stream)

    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None, 0, 0,
                           F.ws_pair)
    once()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    reps = 2
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(reps)]
    for k in range(reps):
        once(evs[k])
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    t_pair = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    t_scr = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    ngq = [len(bse.bse_gvectors(plan, 0, q, 1)) for q in range(nq)]
    flops = sum(8.0 * n * n * dim + iters * 2 * 8.0 * n ** 3 for n in ngq)     # eps GEMM + 2 GEMMs per iteration
    return {"workload": f"{spec.name}, all {nq} q, {iters} Newton-Schulz steps",
            "pair_chi0_ms": t_pair, "screening_ms": t_scr,
            "screening_fp32_tflops": flops / (t_scr / 1e3) / 1e12,
            "newton_schulz_residual_max": float(res.max().item())}


def run_coupled(args, dev, spec, W, om, F, peaks):
    """The BSE with e-h / h-e coupling on the bench workload (A = F.H, P = F.P already built): coupling
    pair densities and the coupling block B over the step's q chunks (FP32 and BF16x3 contractions), and
    the coupled spectrum with 2 nsteps Lanczos steps (its zero-diagonal recursion needs twice the steps of
    the Tamm-Dancoff one for the same resolution).  CUDA-event times; returns the JSON summary."""
    import torch
    from paper_1206_3518_gb300 import bse
    from paper_1206_3518_gb300.pipeline import Coupled

    plan = F.plan
    inf = plan.info(0)
    dim = inf["dim"]
    nsteps = 2 * spec.nsteps
    C = Coupled(F, nsteps=nsteps)
    stream = torch.cuda.current_stream()

    def build(prec, evs=None):
        ev = (lambda: torch.cuda.Event(enable_timing=True)) if evs is not None else None
        marks = []

        def mark():
            if ev:
                e = ev()
                e.record(stream)
                marks.append(e)
        mark()
        bse.bse_build_coupling(plan, 0, bse.BSE_BC_INIT, F.rho_x, None, 0, 0, None, prec, C.Bm, C.ws)
        mark()
        for q0, q1 in F.chunks:
            bse.bse_pair_densities(plan, 0, bse.BSE_PD_COUPLING, None, None, None, None, C.rho_cpl, q0, q1, F.ws_pair)
            mark()
            bse.bse_build_coupling(plan, 0, bse.BSE_BC_DIRECT, None, C.rho_cpl, q0, q1, W, prec, C.Bm, C.ws)
            mark()
        if evs is not None:
            evs.append(marks)

    out = {"workload": f"{spec.name}, dim {dim}, all {inf['nq']} q in {len(F.chunks)} chunks, {nsteps} coupled "
                       f"Lanczos steps", "nsteps": nsteps}
    res = {}
    for name, prec in (("fp32", bse.BSE_PREC_FP32), ("bf16x3", bse.BSE_PREC_BF16X3)):
        build(prec)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        evs = []
        for _ in range(2):
            build(prec, evs)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        init = statistics.mean(m[0].elapsed_time(m[1]) for m in evs)
        pair = statistics.mean(sum(m[1 + 2 * i].elapsed_time(m[2 + 2 * i]) for i in range(len(F.chunks))) for m in evs)
        contract = statistics.mean(sum(m[2 + 2 * i].elapsed_time(m[3 + 2 * i]) for i in range(len(F.chunks)))
                                   for m in evs)
        C.spectrum(om, spec.eta)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        C.spectrum(om, spec.eta)
        e1.record(stream)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        res[name] = C.eps2.clone()
        # the same call replayed from a CUDA graph (6 kernels per Lanczos step, no host launches)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            C.spectrum(om, spec.eta)
        g.replay()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        g.replay()
        g1.record(stream)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        same = bool(torch.equal(res[name], C.eps2))
        del g
        out[name] = {"exchange_init_ms": init, "pair_coupling_ms": pair, "coupling_contract_ms": contract,
                     "spectrum_ms": e0.elapsed_time(e1), "spectrum_graph_ms": g0.elapsed_time(g1),
                     "graph_equals_stream": same, "steps_done": int(C.steps_done.item())}
    t = min(out["fp32"]["spectrum_ms"], out["fp32"]["spectrum_graph_ms"])
    bytes_per_step = 2.0 * dim * dim * 8            # A and B, complex64, once per step
    out["spectrum_hbm_gbs_equiv"] = nsteps * bytes_per_step / (t / 1e3) / 1e9
    out["spectrum_hbm_frac_of_measured"] = out["spectrum_hbm_gbs_equiv"] / peaks["hbm_gbs"] if peaks else None
    out["eps2_bf16x3_rel_err_vs_fp32"] = float((res["bf16x3"] - res["fp32"]).abs().max() / res["fp32"].abs().max())
    out["coupled_spectra_per_s"] = 1e3 / t
    return out


def run_stage(args):
    """One stage alone on the bench workload (for ncu captures); prints per-launch CUDA-event times."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1206_3518_gb300 import bse
    from paper_1206_3518_gb300.pipeline import Forward

    spec, s = make_inputs(args.config)
    plan = bse.Plan([spec])
    qchunk = args.qchunk or (16 if args.only in ("pair", "contract") else 32)
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw, qchunk=qchunk)
    dev = torch.device("cuda")
    coef = torch.as_tensor(s.coef.astype(np.complex64), device=dev)
    en = torch.as_tensor(s.energies, device=dev)
    om = torch.as_tensor(s.omega, device=dev)
    W = torch.as_tensor(s.W, device=dev)
    if args.only == "spectrum":
        F.build(coef, en, W, spec.delta)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, en, F.rho_x, F.P, None, 0, 0,
                           F.ws_pair)
    q0, q1 = F.chunks[min(1, len(F.chunks) - 1)]
    prec = bse.BSE_PREC_BF16X3 if args.prec == "bf16x3" else bse.BSE_PREC_FP32
    if args.only == "contract":
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, en, spec.delta, prec, F.H, None)

    def once():
        if args.only == "pair":
            bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        elif args.only == "contract":
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, W, None, spec.delta, prec, F.H,
                                 F.ws_kernel)
        else:
            F.spectrum(om, spec.eta)

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        once()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    bse.bse_status_read(plan)
    nblk = sum(len(bse.bse_pair_blocks(plan, 0, q)[0]) for q in range(q0, q1)) if args.only != "spectrum" else 0
    print(json.dumps({"stage": args.only, "config": spec.name, "ms": times, "q_range": [q0, q1], "blocks": nblk}))


# DRAM bytes (read + write) of one full-size pair_kernel launch of the fcc 8x8x8 3v4c workload from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, 1 pass), valid while the kernel
# sources hash to the recorded value; see profiles/launches_fcc8x8x8_3v4c_fp32.md.
# DRAM bytes (read + write) of one full-size correlation-kernel launch (direct set, all 512 q), from one ncu
# capture of the sources with this SHA-1 (gcorr.cu + pairjob.cuh); not reported for other sources.
GCORR_TRAFFIC = {"sha1": "a6a9963323c2b537290106ad60bd6e019813b0b5", "bytes": 0.540535296e9 + 7.912874496e9}
PAIR_TRAFFIC = {"sha1": "c39047a0b9675fda883a64bbde1871fdae56455a", "bytes": 101.77e9 + 8.39e9}


def _gcorr_sources_sha1():
    import hashlib
    base = os.path.join(ROOT, "paper_1206_3518_gb300", "csrc")
    data = open(os.path.join(base, "gcorr.cu"), "rb").read() + open(os.path.join(base, "pairjob.cuh"), "rb").read()
    return hashlib.sha1(data).hexdigest()


def _pair_sources_sha1():
    import hashlib
    base = os.path.join(ROOT, "paper_1206_3518_gb300", "csrc")
    data = open(os.path.join(base, "pair.cu"), "rb").read() + open(os.path.join(base, "fft.cuh"), "rb").read()
    return hashlib.sha1(data).hexdigest()


def pair_work(plan, spec, inf):
    """Variant in use for the direct pair densities and, for the plane-wave correlation kernel, its complex
    multiply-adds over all upper blocks: sum_blocks NG(q) |S(k')| (Nv^2 + Nc^2) (the dense (p, G2) loop)."""
    from paper_1206_3518_gb300 import bse
    variants, current = bse.bse_pair_variants(plan, 0)
    v = next(x for x in variants if x["index"] == current)
    if v["rows"] != 0:
        return {"method": "fft", "variant": current}
    npw = [len(bse.bse_gvectors(plan, 0, k, 0)) for k in range(spec.nkpt)]
    cmac = 0
    for q in range(spec.nkpt):
        ng = len(bse.bse_gvectors(plan, 0, q, 1))
        blk, _ = bse.bse_pair_blocks(plan, 0, q)
        cmac += ng * sum(npw[int(k2)] for _, k2 in blk)
    return {"method": "correlation", "variant": current, "cmac": cmac * (spec.nv ** 2 + spec.nc ** 2)}


def roofline(stage, ms, spec, inf, peaks, src, nchunks, pw=None):
    """Algorithmic work of the dominant stage per launch over its measured mean duration."""
    dim = inf["dim"]
    nb = inf["nblocks"]
    n1, n2, n3 = spec.fft
    if stage == "pair_direct" and pw and pw["method"] == "correlation":
        flops = 8.0 * pw["cmac"] / nchunks
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = flops / (ms / 1e3) / 1e12
        return {"bound": "alu", "kernel": "gcorr_kernel", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak,
                "work": "8 FP32 flops per complex multiply-add of the plane-wave correlation's (G, G2) loop: "
                        "sum over blocks of NG(q) |S(k')| (Nv^2 + Nc^2)",
                "traffic": (GCORR_TRAFFIC["bytes"] if nchunks == 1 and spec.name == "fcc_8x8x8_3v4c"
                            and _gcorr_sources_sha1() == GCORR_TRAFFIC["sha1"] else None),
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock"}
    if stage == "pair_direct":
        import math
        nr = n1 * n2 * n3
        products = nb * (spec.nv ** 2 + spec.nc ** 2)
        flops = products * 5.0 * nr * math.log2(nr) / nchunks
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"bound": "alu", "kernel": "pair_kernel", "achieved": flops / (ms / 1e3) / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak,
                "work": "5 N_r log2 N_r FP32 flops per pair-density FFT (FFT convention)",
                "traffic": (PAIR_TRAFFIC["bytes"] if nchunks == 1 and spec.name == "fcc_8x8x8_3v4c"
                            and _pair_sources_sha1() == PAIR_TRAFFIC["sha1"] else None),
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock"}
    if stage == "spectrum":
        bytes_ = spec.nsteps * 8.0 * dim * dim
        ach = bytes_ / (ms / 1e3) / 1e9
        return {"bound": "hbm", "kernel": "haydock_kernel", "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "work": "8 dim^2 bytes of H per Haydock step",
                "traffic": None, "peak_source": src}
    if stage == "direct_contract":
        w = min(spec.nv ** 2, spec.nc ** 2)
        ng = inf["ng_max"]
        flops = 8.0 * (nb * w * ng * ng + nb * spec.nv ** 2 * spec.nc ** 2 * ng) / nchunks
        ach = flops / (ms / 1e3) / 1e12
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        return {"bound": "alu", "kernel": "gemm_wr", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "work": "8 flops per complex MAC of W.R and the block products",
                "traffic": None, "peak_source": "derived FP32 CUDA-core peak"}
    return {"bound": "hbm", "kernel": stage, "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": None, "traffic": None}


def cpu_baseline(spec, s, budget_s=20.0):
    """The oracle as it stands on the host cores, on a bounded sample scaled to one full step."""
    import numpy as np
    import time as _t
    from oracle import geometry as geo, kernel as ok, pair as op, spectrum as osp
    cores = os.cpu_count()
    blocks = geo.upper_blocks(spec)
    rng = np.random.default_rng(0)
    t0 = _t.perf_counter()
    nsample = 0
    for idx in rng.permutation(len(blocks)):
        ik, ik2 = blocks[idx]
        iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
        ok.direct_block(spec, rv, rc, ok.w_of_q(spec, s.W, iq))
        nsample += 1
        if _t.perf_counter() - t0 > 0.6 * budget_s:
            break
    t_block = (_t.perf_counter() - t0) / nsample
    # Haydock: a few steps of the oracle recursion on a dense Hermitian matrix of the same size
    dim = spec.dim
    m = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))).astype(np.complex128)
    Hs = 0.5 * (m + m.conj().T)
    P = rng.standard_normal(dim) + 0j
    nst = 4
    t1 = _t.perf_counter()
    osp.haydock(Hs, P, nst)
    t_hay = (_t.perf_counter() - t1) / nst
    t_step = t_block * len(blocks) + t_hay * spec.nsteps
    return {"value": dim * dim / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nsample} random upper (k,k') blocks (pair densities by correlation + K^d) and {nst} Haydock "
                      f"steps at dim {dim}, scaled to {len(blocks)} blocks + {spec.nsteps} steps",
            "est_step_s": t_step}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, s = make_inputs(args.config)
    times = []
    base = None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        base = cpu_baseline(spec, s, budget_s=args.cpu_budget)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    from oracle import geometry as geo
    ng_max = max(len(geo.sphere(spec, tuple(o))) for o in geo.mesh_offsets(spec))
    out = {"metric": METRIC, "value": base["value"], "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": base["est_step_s"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": dict(workload_config(spec, ng_max), precision="complex128 oracle (CPU), bounded sample per step",
                          parallelism="host cores"),
           "cpu_baseline": {"kind": "oracle", "cores": base["cores"], "sample": base["sample"], "value": base["value"]},
           "e2e": {"value": base["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="fcc_8x8x8_3v4c")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the BF16x3 comparison run")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch of hexagonal sheets")
    ap.add_argument("--no-screening", action="store_true", help="skip the static RPA screening measurement")
    ap.add_argument("--no-coupled", action="store_true", help="skip the BSE with e-h / h-e coupling")
    ap.add_argument("--only", default="all", choices=["all", "pair", "spectrum", "contract"],
                    help="profiling aid: run one stage (pair: realspace + a q chunk of pair densities; "
                         "spectrum: Haydock on an H built once before the loop)")
    ap.add_argument("--qchunk", type=int, default=0, help="q points per direct-term chunk (0 = all)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only != "all":
        run_stage(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
