"""Benchmark of the BSE hot path: one step = pair densities + Hamiltonian + Haydock spectrum.

Headline workload: fcc 12x12x12 k mesh, 4 valence + 4 conduction bands (dim 27648),
~496 plane waves per sphere (max 531), 48^3 grid, 300 Haydock steps, 2000
frequencies, eta 0.05 eV (synthetic inputs of the paper's 12x12x12 convergence
shape, Sec. IV C).  The step runs twice on the same inputs: with FP32 contractions
and with BF16 hi/lo split-complex tensor-core contractions ("mixed", FP32
accumulation); ``value`` is the mixed step's kernel elements/s (dim^2 per step) and
the FP32 step is reported beside it.  The direct pair densities (203 GB over all q)
and the W.rho products are streamed in q chunks.  Every input (u store 12.3 GB,
H 6.1 GB, W 3.9 GB) is larger than the 129 MB L2, so no flush is needed between
steps.  Multi-GPU runs are independent replicas (weak scaling).

Secondary measurements on fcc 8x8x8 3v4c (dim 6144): static RPA screening, the BSE
with e-h/h-e coupling, the q-point symmetry reduction of W, and the batch of 16
hexagonal sheets.

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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("BSE kernel elements/s (dim^2 per full step: pair densities + H + Haydock eps_2), mixed (BF16x3 "
          "tensor-core contractions) vs FP32, eps_2 within 1e-3 of the FP64 oracle")
UNIT = "elements/s"
HEADLINE = "fcc_12x12x12_4v4c"
SECONDARY = "fcc_8x8x8_3v4c"
STAGES = ["realspace+exchange", "exchange_kernel", "pair_direct", "direct_contract", "spectrum"]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (the samples go to a temporary file)."""

    def __init__(self):
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="bse_clocks_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
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
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
                power.append(float(p[3]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "power_w_max": max(power) if power else None, "samples": len(sm)}


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


def workload_config(spec, ng_max, qchunk=None, nchunks=None):
    """The workload description shared by both arms of the bench."""
    lat = "fcc a=10 bohr" if spec.lattice == "fcc" else f"hex a={spec.a} c={spec.c} bohr"
    u_gb = spec.nkpt * spec.nb * spec.fft[0] * spec.fft[1] * spec.fft[2] * 8 / 1e9
    h_gb = spec.dim * spec.dim * 8 / 1e9
    w_gb = spec.nkpt * ng_max * ng_max * 8 / 1e9
    out = {"workload": f"{spec.name}: {lat}, {spec.nk[0]}x{spec.nk[1]}x{spec.nk[2]} k, {spec.nv}v{spec.nc}c, "
                       f"dim {spec.dim}, Ecut {spec.ecut} Ha (ng_max {ng_max}), grid "
                       f"{spec.fft[0]}x{spec.fft[1]}x{spec.fft[2]}, {spec.nsteps} Haydock steps, {spec.nw} w",
           "dim": spec.dim, "nblocks": spec.nkpt * (spec.nkpt + 1) // 2,
           "l2": f"inputs larger than L2 (u {u_gb:.2f} GB, H {h_gb:.2f} GB, W {w_gb:.2f} GB); no flush"}
    if qchunk is not None:
        out["q_chunk"] = qchunk
        out["q_chunks"] = nchunks
    return out


def make_inputs(name):
    from synth import config_spec, generate
    import numpy as np
    spec = config_spec(name)
    s = generate(spec, wdtype=np.complex64)
    return spec, s


def auto_qchunk(plan, nq, budget_bytes, align=1):
    """Fewest q chunks whose direct pair densities and W.rho workspace fit in budget_bytes; with align > 1
    the chunk is rounded down to a multiple of align (whole planes of the q mesh, so that the tensor-core
    pair route sees whole planes of k' for every k and fills its regions)."""
    from paper_1206_3518_gb300 import bse
    for n in range(1, nq + 1):
        ch = -(-nq // n)
        if align > 1 and ch > align:
            ch = ch // align * align
        chunks = [(q, min(q + ch, nq)) for q in range(0, nq, ch)]
        rho = max(bse.bse_rho_dir_count(plan, 0, a, b) for a, b in chunks) * plan.info(0)["ng_max"] * 8
        ws = bse.bse_workspace_size(plan, 0, bse.BSE_WS_KERNEL, ch)
        if rho + ws <= budget_bytes:
            return ch
    return 1


class Step:
    """One full step of the hot path (A1-A8) on preallocated buffers, with optional per-stage events."""

    def __init__(self, plan, F, spec, coef, en, W, om, stream):
        self.plan, self.F, self.spec = plan, F, spec
        self.coef, self.en, self.W, self.om = coef, en, W, om
        self.stream = stream
        self.launches = 0

    def __call__(self, prec, marks=None, w_ready=None, w_free=None):
        """w_ready / w_free (end to end): per q chunk, the event after which that chunk's rows of W are on the
        device, and the event this step records once its direct term has read them."""
        import torch
        from paper_1206_3518_gb300 import bse
        F, spec, plan = self.F, self.spec, self.plan

        def mark(label):
            if marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(self.stream)
                marks.append((label, e))
        mark(None)
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, self.coef, self.en, F.rho_x,
                               F.P, None, 0, 0, F.ws_pair)
        mark("realspace+exchange")
        bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, self.en, spec.delta, prec, F.H,
                             F.ws_kernel if prec == bse.BSE_PREC_BF16X3 else None)
        mark("exchange_kernel")
        fdir = bse.BSE_PD_DIRECT | (bse.BSE_PD_TENSOR if self.tensor_pair(prec) else 0)
        for c, (q0, q1) in enumerate(F.chunks):
            bse.bse_pair_densities(plan, 0, fdir, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
            mark("pair_direct")
            if w_ready is not None:
                self.stream.wait_event(w_ready[c])
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, self.W, None, spec.delta, prec,
                                 F.H, F.ws_kernel)
            if w_free is not None:
                w_free[c].record(self.stream)
            mark("direct_contract")
        bse.bse_spectrum(plan, 0, F.H, F.P, spec.nsteps, self.om, spec.eta, F.eps2, F.ab, F.steps_done, F.ws_spec)
        mark("spectrum")

    def tensor_pair(self, prec):
        """The mixed step takes the direct pair densities on the tensor cores where the system has that route."""
        from paper_1206_3518_gb300 import bse
        return prec == bse.BSE_PREC_BF16X3 and bool(self.F.info["tensor_pair"])

    def kernels_per_step(self, prec):
        """Kernel launches of one step: realspace, exchange densities, dipole, K^x (BF16x3: operand split and
        Gram kernel); per chunk the direct densities (FP32: the correlation kernel; BF16x3: image packing, tile
        table and the tcgen05 kernel, plus the FP64 G = 0 overlaps on the chunk holding q = 0) and the direct
        term (FP32: W.rho GEMM + block kernel; BF16x3: two operand splits, the tcgen05 GEMM and the block
        kernel); the Haydock kernel."""
        from paper_1206_3518_gb300 import bse
        mixed = prec == bse.BSE_PREC_BF16X3
        pair = 3 if self.tensor_pair(prec) else 1
        per_chunk = pair + (4 if mixed else 2)
        return 4 + (1 if mixed else 0) + per_chunk * len(self.F.chunks) + (1 if self.tensor_pair(prec) else 0) + 1


def stage_times(marks_per_step):
    """Mean milliseconds per stage over the timed steps (an interval belongs to the label of its end)."""
    out = {n: 0.0 for n in STAGES}
    for marks in marks_per_step:
        for (_, a), (lab, b) in zip(marks[:-1], marks[1:]):
            out[lab] += a.elapsed_time(b)
    return {n: v / len(marks_per_step) for n, v in out.items()}


def timed_loop(step, prec, steps, warmup, world, dev):
    """W untimed steps, then K steps bracketed by a barrier and synchronisations; returns (ms/step, stages)."""
    import torch
    import torch.distributed as dist
    for _ in range(warmup):
        step(prec)
    torch.cuda.synchronize()
    marks = [[] for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(step.stream)
    for k in range(steps):
        step(prec, marks[k])
    t1.record(step.stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dev) / steps
    return ms, stage_times(marks)


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
    free, _ = torch.cuda.mem_get_info(dev)
    fixed = (bse.bse_workspace_size(plan, 0, bse.BSE_WS_PAIR) + 2 * dim * dim * 8
             + inf["nq"] * inf["ng_max"] ** 2 * 8 * 2)
    plane = spec.nk[1] * spec.nk[2] if inf["tensor_pair"] else 1
    qchunk = args.qchunk or auto_qchunk(plan, inf["nq"], int(0.6 * (free - fixed)), plane)
    F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw, qchunk=qchunk)
    coef_h = torch.as_tensor(s.coef.astype(np.complex64)).pin_memory()
    en_h = torch.as_tensor(s.energies).pin_memory()
    W_h = torch.as_tensor(s.W).pin_memory()
    om_h = torch.as_tensor(s.omega).pin_memory()
    coef, en, W, om = (coef_h.to(dev), en_h.to(dev), W_h.to(dev), om_h.to(dev))
    stream = torch.cuda.current_stream()
    step = Step(plan, F, spec, coef, en, W, om, stream)
    FP32, MIXED = bse.BSE_PREC_FP32, bse.BSE_PREC_BF16X3

    clocks = Clocks()
    clocks.start()
    ms32, st32 = timed_loop(step, FP32, args.steps, args.warmup, world, dev)
    bse.bse_status_read(plan)
    eps32 = F.eps2.clone()
    steps32 = int(F.steps_done.item())
    H32 = F.H.cpu().numpy() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    msmx, stmx = timed_loop(step, MIXED, args.steps, args.warmup, world, dev)
    ck = clocks.stop()
    bse.bse_status_read(plan)
    epsmx = F.eps2.clone()
    Hmx = F.H.cpu().numpy() if H32 is not None else None

    # end to end through host buffers at the headline (mixed) precision: inputs H2D from pinned memory and
    # eps_2 D2H every step.  W (the largest input) is uploaded on a second stream, one q chunk's rows at a
    # time: chunk c's rows as soon as the previous step's direct term of chunk c has read them, and the
    # direct term of chunk c waits for its own rows only.
    eps_host = torch.empty(spec.nw, dtype=torch.float64).pin_memory()
    h2d = coef_h.numel() * 8 + en_h.numel() * 8 + W_h.numel() * 8 + om_h.numel() * 8
    d2h = spec.nw * 8
    e_steps = max(1, min(args.steps, 3))
    side = torch.cuda.Stream()
    w_free = [torch.cuda.Event() for _ in F.chunks]
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for ev in w_free:
        ev.record(stream)
    for _ in range(e_steps):
        coef.copy_(coef_h, non_blocking=True)
        en.copy_(en_h, non_blocking=True)
        om.copy_(om_h, non_blocking=True)
        w_ready = []
        for c, (q0, q1) in enumerate(F.chunks):
            side.wait_event(w_free[c])
            with torch.cuda.stream(side):
                W[q0:q1].copy_(W_h[q0:q1], non_blocking=True)
            w_ready.append(torch.cuda.Event())
            w_ready[-1].record(side)
        step(MIXED, w_ready=w_ready, w_free=w_free)
        eps_host.copy_(F.eps2, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e_steps, world, dev)
    e2e_same = bool(np.array_equal(eps_host.numpy(), epsmx.cpu().numpy()))

    peaks, src = _peaks()
    pw = pair_work(plan, spec, inf)
    roofs32 = stage_rooflines(st32, spec, inf, peaks, src, len(F.chunks), pw, FP32)
    roofsmx = stage_rooflines(stmx, spec, inf, peaks, src, len(F.chunks), pw, MIXED)
    dom = max(stmx, key=stmx.get)
    e32 = eps32.cpu().numpy()
    emx = epsmx.cpu().numpy()
    kernel_only = lambda ms, st: dim * dim / ((ms - st["spectrum"]) / 1e3)  # noqa: E731
    out = {
        "metric": METRIC, "value": world * dim * dim / (msmx / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": msmx, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": dict(workload_config(spec, inf["ng_max"], qchunk, len(F.chunks)),
                       precision="headline: BF16 hi/lo split-complex tcgen05 contractions (direct pair "
                                 "densities, K^x and W.rho), FP32 exchange densities and block products, FP64 "
                                 "G = 0 overlaps, Lanczos coefficients and continued fraction; compared with "
                                 "the all-FP32 step",
                       parallelism=f"replicas x{world}"),
        "stages_ms": stmx,
        "kernel_elements_per_s": kernel_only(msmx, stmx),
        "spectra_per_s": 1e3 / stmx["spectrum"],
        "fp32": {"value": world * dim * dim / (ms32 / 1e3), "ms_per_step": ms32, "stages_ms": st32,
                 "kernel_elements_per_s": kernel_only(ms32, st32), "spectra_per_s": 1e3 / st32["spectrum"],
                 "stage_rooflines": roofs32, "steps_done": steps32},
        "mixed_over_fp32": ms32 / msmx,
        "eps2_mixed_rel_err_vs_fp32": float(np.abs(emx - e32).max() / np.abs(e32).max()),
        "roofline": roofsmx[dom],
        "stage_rooflines": roofsmx,
        "clocks": ck,
        "e2e": {"value": world * dim * dim / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "prec": "bf16x3", "eps2_equals_device_run": e2e_same},
        "gpu_launches": args.steps * (step.kernels_per_step(FP32) + step.kernels_per_step(MIXED)),
        "gpu_launches_note": "both timed loops (FP32 and mixed), K steps each",
    }
    if H32 is not None:
        out["cpu_baseline"] = cpu_baseline(spec, s, H32, Hmx, e32, emx, steps32, budget_s=args.cpu_budget)
        out["cpu_baseline"]["full_small"] = cpu_full_small()
        del H32, Hmx

    del F, step, coef, en, W, om, coef_h, W_h
    torch.cuda.empty_cache()
    if not args.no_secondary:
        out["secondary"] = run_secondary(args, dev, rank, world, peaks)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def run_secondary(args, dev, rank, world, peaks):
    """The rows beyond the TDA step on fcc 8x8x8 3v4c (dim 6144) and the batch of sheets."""
    import numpy as np
    import torch
    from paper_1206_3518_gb300 import bse
    from paper_1206_3518_gb300.pipeline import Forward

    out = {}
    if world == 1 and not (args.no_screening and args.no_coupled and args.no_symmetry and args.no_tddft and
                           args.no_states):
        spec, s = make_inputs(SECONDARY)
        plan = bse.Plan([spec])
        inf = plan.info(0)
        F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
        coef = torch.as_tensor(s.coef.astype(np.complex64), device=dev)
        en = torch.as_tensor(s.energies, device=dev)
        W = torch.as_tensor(s.W, device=dev)
        om = torch.as_tensor(s.omega, device=dev)
        F.build(coef, en, W, spec.delta)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        if not args.no_screening:
            out["screening"] = run_screening(args, dev, spec, s, coef, en, F)
            F.build(coef, en, W, spec.delta)
        if not args.no_symmetry:
            out["symmetry"] = run_symmetry(plan, inf, W, dev)
        if not args.no_coupled:
            out["coupled"] = run_coupled(args, dev, spec, W, om, F, peaks)
        if not args.no_tddft:
            out["tddft"] = run_tddft(args, dev, spec, s, en, F, peaks)
        if not args.no_states:
            F.build(coef, en, W, spec.delta)
            out["exciton_states"] = run_states(dev, spec, F, peaks)
        del F, coef, en, W, om
        torch.cuda.empty_cache()
    if world == 1 and not args.no_symmetry:
        out["kpoint_symmetry"] = run_kpoint_symmetry(dev)
    if not args.no_batch:
        out["batch"] = run_batch(args, dev, rank, world)
    return out


def run_kpoint_symmetry(dev):
    """k-point symmetry of the blocks (Sec. III A) on fcc 8x8x8 3v4c with states that carry the point group
    and a diagonal model W: the build of every upper block against the build of the representatives plus
    the fill stage, on the same inputs; CUDA-event times, H and eps_2 differences."""
    import numpy as np
    import torch
    from paper_1206_3518_gb300 import bse
    from paper_1206_3518_gb300.pipeline import Forward
    from synth import config_spec, generate
    spec = config_spec(SECONDARY).replace(name="fcc_8x8x8_3v4c_symmetric", symmetric=True, w_offdiag=0.0)
    s = generate(spec, wdtype=np.complex64)
    coef = torch.as_tensor(s.coef.astype(np.complex64), device=dev)
    en = torch.as_tensor(s.energies, device=dev)
    W = torch.as_tensor(s.W, device=dev)
    om = torch.as_tensor(s.omega, device=dev)
    res = {}
    for label, sym_on in (("full", False), ("reduced", True)):
        plan = bse.Plan([spec.replace(symmetric=sym_on)])
        inf = plan.info(0)
        F = Forward(plan, 0, nsteps=spec.nsteps, nw=spec.nw)
        F.build(coef, en, W, spec.delta)
        torch.cuda.synchronize()
        bse.bse_status_read(plan)
        times = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            F.build(coef, en, W, spec.delta)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        eps = F.spectrum(om, spec.eta).cpu().numpy().copy()
        bse.bse_status_read(plan)
        res[label] = {"build_ms": statistics.mean(times), "blocks_built": inf["nblocks"], "H": F.H.cpu().numpy(),
                      "eps": eps}
        del F, plan
        torch.cuda.empty_cache()
    dh = float(np.abs(res["reduced"]["H"] - res["full"]["H"]).max() / np.abs(res["full"]["H"]).max())
    de = float(np.abs(res["reduced"]["eps"] - res["full"]["eps"]).max() / np.abs(res["full"]["eps"]).max())
    return {"workload": f"{spec.name}: states carrying the 48 operations of the point group, diagonal model W",
            "blocks_full": res["full"]["blocks_built"], "blocks_reduced": res["reduced"]["blocks_built"],
            "build_ms_full": res["full"]["build_ms"], "build_ms_reduced": res["reduced"]["build_ms"],
            "speedup": res["full"]["build_ms"] / res["reduced"]["build_ms"],
            "H_rel_diff": dh, "eps2_rel_diff": de}


def run_tddft(args, dev, spec, s, en, F, peaks):
    """Macroscopic dielectric function from TDDFT with local fields on the workload's frequency grid: the
    optical-limit Adler-Wiser response chi~0(w) for every frequency, the ALDA kernel and the Dyson solve with
    RPA and ALDA kernels (eps_M = 1/[eps^-1]_00).  CUDA-event times; returns the JSON summary."""
    import torch
    from paper_1206_3518_gb300 import bse
    plan = F.plan
    inf = plan.info(0)
    ng, dim, nw = inf["ng0"], inf["dim"], spec.nw
    omega = torch.as_tensor(s.omega, device=dev)
    bse.bse_pair_densities(plan, 0, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, torch.as_tensor(
        s.coef.astype("complex64"), device=dev), en, F.rho_x, F.P, None, 0, 0, F.ws_pair)
    chi = torch.empty(nw, ng, ng, dtype=torch.complex64, device=dev)
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_CHI0) // 8 + 1, dtype=torch.complex64, device=dev)
    Fx = torch.empty(ng, ng, dtype=torch.complex64, device=dev)
    wsa = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_ALDA) // 8 + 1, dtype=torch.complex64, device=dev)
    wse = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_EPSM, nw) // 8 + 1, dtype=torch.complex64,
                      device=dev)
    e_rpa = torch.empty(nw, dtype=torch.complex128, device=dev)
    e_alda = torch.empty(nw, dtype=torch.complex128, device=dev)
    eta = spec.eta

    def once(ev=None):
        marks = []

        def mark():
            if ev is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                marks.append(e)
        mark()
        bse.bse_chi0_optical(plan, 0, F.rho_x, F.P, en, spec.delta, omega, eta, chi, ws)
        mark()
        bse.bse_xc_kernel_alda(plan, 0, F.ws_pair, Fx, wsa)
        mark()
        bse.bse_epsilon_macro(plan, 0, chi, None, e_rpa, wse)
        mark()
        bse.bse_epsilon_macro(plan, 0, chi, Fx, e_alda, wse)
        mark()
        if ev is not None:
            ev.append(marks)

    once()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    evs = []
    for _ in range(2):
        once(evs)
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    t = [statistics.mean(m[i].elapsed_time(m[i + 1]) for m in evs) for i in range(4)]
    flops = 2.0 * 8.0 * nw * ng * ng * dim            # two weighted Gram terms, 8 flops per complex MAC
    ach = flops / (t[0] / 1e3) / 1e12
    fp32 = _fp32_peak(peaks)
    er = e_rpa.cpu().numpy()
    ea = e_alda.cpu().numpy()
    i = int(abs(s.omega).argmin())
    return {"workload": f"{spec.name}, q -> 0 sphere of {ng} G, {dim} transitions, {nw} w, eta {eta:.4f} Ha",
            "chi0_ms": t[0], "alda_kernel_ms": t[1], "eps_m_rpa_ms": t[2], "eps_m_alda_ms": t[3],
            "chi0_roofline": {"bound": "alu", "kernel": "chi0_kernel", "achieved": ach, "peak": fp32,
                              "unit": "TFLOP/s", "frac": ach / fp32,
                              "work": "2 x 8 FP32 flops per complex MAC of nw ng0^2 dim"},
            "eps_m_static_rpa": float(er[i].real), "eps_m_static_alda": float(ea[i].real),
            "static_frequency_ha": float(s.omega[i])}


def run_states(dev, spec, F, peaks):
    """All eigenpairs of the workload's H (Eq. bse_eig) by the full-dimension Lanczos tridiagonalisation,
    bisection, inverse iteration and back-transformation; CUDA-event time and the residual of the pairs."""
    import numpy as np
    import torch
    from paper_1206_3518_gb300 import bse
    plan = F.plan
    dim = F.dim
    n = dim
    rng = np.random.default_rng(5)
    x0 = torch.as_tensor(rng.standard_normal(dim) + 1j * rng.standard_normal(dim), device=dev)
    theta = torch.empty(n, dtype=torch.float64, device=dev)
    A = torch.empty(n, dim, dtype=torch.complex64, device=dev)
    ab = torch.empty(2 * n, dtype=torch.float64, device=dev)
    done = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(bse.bse_workspace_size(plan, 0, bse.BSE_WS_STATES, n) // 8 + 1, dtype=torch.complex64,
                     device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    bse.bse_exciton_states(plan, 0, F.H, x0, n, theta, A, ab, done, ws)
    e1.record()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    ms = e0.elapsed_time(e1)
    # residual |H A_l - theta_l A_l| / |H| on a sample of 64 states (row products on the device)
    idx = torch.as_tensor(np.linspace(0, n - 1, 64).astype(np.int64), device=dev)
    As = A[idx]
    R = As @ F.H.transpose(0, 1) - theta[idx].to(torch.complex64)[:, None] * As
    res = float(R.abs().max() / F.H.abs().max())
    h_bytes = float(n) * 8.0 * dim * dim
    return {"workload": f"{spec.name}, all {n} eigenpairs from a random start vector", "ms": ms,
            "steps_done": int(done.item()), "residual_max_64_sampled": res,
            "lanczos_h_stream_gbs_lower_bound": h_bytes / (ms / 1e3) / 1e9}


def run_symmetry(plan, inf, W, dev):
    """q-point symmetry (Sec. III A): W of the irreducible points only, unfolded on the device."""
    import numpy as np
    import torch
    from paper_1206_3518_gb300 import bse
    nops, ibz_q, _, _ = bse.bse_symmetry(plan, 0)
    W_ibz = W[torch.as_tensor(ibz_q.astype(np.int64), device=dev)].contiguous()
    W_full = torch.empty_like(W)
    bse.bse_unfold_w(plan, 0, W_ibz, W_full, 0, inf["nq"])
    torch.cuda.synchronize()
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record()
    bse.bse_unfold_w(plan, 0, W_ibz, W_full, 0, inf["nq"])
    u1.record()
    torch.cuda.synchronize()
    bse.bse_status_read(plan)
    return {"ops": nops, "irreducible_q": int(len(ibz_q)), "q": inf["nq"], "w_bytes_irreducible": W_ibz.numel() * 8,
            "w_bytes_full": W.numel() * 8, "unfold_ms": u0.elapsed_time(u1)}


def run_batch(args, dev, rank=0, world=1):
    """Layered 2D batch: 16 hexagonal sheets (dims 576..20736), BF16x3 contractions, autotuned pair tiles
    (the tensor-core route of the direct densities among the candidates),
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
        r = autotune.tune(plan, i, F, with_tensor=True)
        tuned.append("tensor" if r.get("tensor") else r["variant"]["index"])
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

    from synth import config_spec, generate
    spec = config_spec(args.config)
    if args.nk:
        spec = spec.replace(nk=(args.nk,) * 3)
    s = generate(spec, wdtype=np.complex64)
    plan = bse.Plan([spec])
    if args.variant >= 0:
        bse.bse_set_pair_variant(plan, 0, args.variant)
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
    ws_init = F.ws_kernel if prec == bse.BSE_PREC_BF16X3 else None
    if args.only == "contract":
        bse.bse_pair_densities(plan, 0, bse.BSE_PD_DIRECT, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, en, spec.delta, prec, F.H, ws_init)

    fdir = bse.BSE_PD_DIRECT | (bse.BSE_PD_TENSOR if prec == bse.BSE_PREC_BF16X3 and F.info["tensor_pair"] else 0)

    def once():
        if args.only == "pair":
            bse.bse_pair_densities(plan, 0, fdir, None, None, None, None, F.rho_dir, q0, q1, F.ws_pair)
        elif args.only == "contract":
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_DIRECT, None, F.rho_dir, q0, q1, W, None, spec.delta, prec, F.H,
                                 F.ws_kernel)
        elif args.only == "exchange":
            bse.bse_build_kernel(plan, 0, bse.BSE_BK_INIT, F.rho_x, None, 0, 0, None, en, spec.delta, prec, F.H,
                                 ws_init)
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
    nblk = (sum(len(bse.bse_pair_blocks(plan, 0, q)[0]) for q in range(q0, q1))
            if args.only in ("pair", "contract") else 0)
    print(json.dumps({"stage": args.only, "config": spec.name, "ms": times, "q_range": [q0, q1], "blocks": nblk}))



# DRAM bytes (read + write) per upper block of the correlation kernel's direct set (the default schedule,
# gcorr_kernel<4, 4, 1, 0>), from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one launch) of
# the fcc 12x12x12 4v4c block shape (Ecut 12, 48^3 grid) on a 6x6x6 k mesh: 23,436 blocks (all 216 q) in one
# launch, 4.5 GB on the device, 155.8 MB read and 2939.5 MB written.  A full launch of the workload processes
# nblocks / q_chunks blocks of the same shape and the bytes grow with the blocks (the densities are written
# once, the coefficients are read from L2), so the traffic per launch is this figure times the launch's
# blocks.  Valid only for the sources with this SHA-1 (gcorr.cu + pairjob.cuh) and that block shape.
GCORR_TRAFFIC = {"sha1": "ebbbbf8406f12035e2778354e7d61fd0fc693ec8", "bytes_per_block": 132074.1,
                 "shape": ("fcc", 4, 4, 12.0)}


# The same for the tensor-core route's kernel (tcpair_kernel): one ncu capture (--set full, one launch) of
# the fcc 12x12x12 4v4c block shape on a 6x6x6 k mesh, q 72..144 (two whole planes of the q mesh, as the
# bench's chunks are): 9,072 blocks, 357.2 MB read and 1415.1 MB written (the densities at their sphere
# positions; the region panels of B mostly from L2).  Valid only for the sources with this SHA-1
# (tcpair.cu + umma.cuh) and that block shape.
TCPAIR_TRAFFIC = {"sha1": "44be08bd79adb79e5e4217dbf94880d38196fef7", "bytes_per_block": 195365.4,
                  "shape": ("fcc", 4, 4, 12.0)}


def _tcpair_sources_sha1():
    import hashlib
    base = os.path.join(ROOT, "paper_1206_3518_gb300", "csrc")
    data = open(os.path.join(base, "tcpair.cu"), "rb").read() + open(os.path.join(base, "umma.cuh"), "rb").read()
    return hashlib.sha1(data).hexdigest()


def _gcorr_sources_sha1():
    import hashlib
    base = os.path.join(ROOT, "paper_1206_3518_gb300", "csrc")
    data = open(os.path.join(base, "gcorr.cu"), "rb").read() + open(os.path.join(base, "pairjob.cuh"), "rb").read()
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
    return {"method": "correlation", "variant": current, "cmac": cmac * (spec.nv ** 2 + spec.nc ** 2),
            "tensor": bool(inf["tensor_pair"])}


def _fp32_peak(peaks):
    return 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def stage_rooflines(st, spec, inf, peaks, src, nchunks, pw, prec):
    """Per stage: algorithmic work of one step (the sum over the stage's launches) over the stage's measured
    time in the step; ``achieved`` is therefore the mean over its launches."""
    import math
    dim, nb, ng = inf["dim"], inf["nblocks"], inf["ng_max"]
    fp32 = _fp32_peak(peaks)
    out = {}
    ms = st["pair_direct"]
    if prec != 0 and pw.get("tensor"):
        useful = 24.0 * pw["cmac"]
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        same = (TCPAIR_TRAFFIC["shape"] == (spec.lattice, spec.nv, spec.nc, spec.ecut)
                and TCPAIR_TRAFFIC["sha1"] == _tcpair_sources_sha1())
        out["pair_direct"] = {
            "bound": "tensor", "kernel": "tcpair_kernel", "achieved": useful / (ms / 1e3) / 1e12, "peak": peak,
            "unit": "TFLOP/s", "frac": useful / (ms / 1e3) / 1e12 / peak, "launches_per_step": 3 * nchunks + 1,
            "work": "BF16x3 split-complex flops of the correlation itself: 3 hi/lo products x 8 real flops per "
                    "complex multiply-add, sum over upper blocks of NG(q) |S(k')| (Nv^2 + Nc^2) (the padding of "
                    "a tile's rows and K positions to the union of its spheres is not counted); the stage's "
                    "whole time (image packing and tile table included)",
            "traffic": TCPAIR_TRAFFIC["bytes_per_block"] * nb / nchunks if same else None,
            "peak_source": src + " (sustained bf16: timed inside a long step)"}
    elif pw["method"] == "correlation":
        flops = 8.0 * pw["cmac"]
        same = (GCORR_TRAFFIC["shape"] == (spec.lattice, spec.nv, spec.nc, spec.ecut)
                and GCORR_TRAFFIC["sha1"] == _gcorr_sources_sha1())
        traffic = GCORR_TRAFFIC["bytes_per_block"] * nb / nchunks if same else None
        out["pair_direct"] = {
            "bound": "alu", "kernel": "gcorr_kernel", "achieved": flops / (ms / 1e3) / 1e12, "peak": fp32,
            "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / fp32, "launches_per_step": nchunks,
            "work": "8 FP32 flops per complex multiply-add of the plane-wave correlation's (G, G2) loop: sum "
                    "over upper blocks of NG(q) |S(k')| (Nv^2 + Nc^2)",
            "traffic": traffic, "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock"}
    else:
        nr = spec.fft[0] * spec.fft[1] * spec.fft[2]
        flops = nb * (spec.nv ** 2 + spec.nc ** 2) * 5.0 * nr * math.log2(nr)
        out["pair_direct"] = {
            "bound": "alu", "kernel": "pair_kernel", "achieved": flops / (ms / 1e3) / 1e12, "peak": fp32,
            "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / fp32, "launches_per_step": nchunks,
            "work": "5 N_r log2 N_r FP32 flops per pair-density FFT (FFT convention)", "traffic": None,
            "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x max SM clock"}
    ms = st["spectrum"]
    bytes_ = spec.nsteps * 8.0 * dim * dim
    out["spectrum"] = {"bound": "hbm", "kernel": "haydock_kernel", "achieved": bytes_ / (ms / 1e3) / 1e9,
                       "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": bytes_ / (ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                       "work": "8 dim^2 bytes of H per Haydock step", "traffic": None, "peak_source": src,
                       "launches_per_step": 1}
    ms = st["direct_contract"]
    w = min(spec.nv ** 2, spec.nc ** 2)
    cmac_wr = float(nb) * w * ng * ng
    cmac_blk = float(nb) * spec.nv ** 2 * spec.nc ** 2 * ng
    if prec == 0:
        flops = 8.0 * (cmac_wr + cmac_blk)
        out["direct_contract"] = {
            "bound": "alu", "kernel": "gemm_wr + block_kernel", "achieved": flops / (ms / 1e3) / 1e12, "peak": fp32,
            "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / fp32, "launches_per_step": 2 * nchunks,
            "work": "8 flops per complex MAC of W.R (ng_max^2 min(Nv^2, Nc^2) per block) and the block products",
            "traffic": None, "peak_source": "derived FP32 CUDA-core peak"}
    else:
        issued = 24.0 * cmac_wr
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        out["direct_contract"] = {
            "bound": "tensor", "kernel": "split_a/split_b + tc_gemm_wr + block_kernel",
            "achieved": issued / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": issued / (ms / 1e3) / 1e12 / peak, "launches_per_step": 4 * nchunks,
            "work": "issued BF16 MMA flops of W.R: 3 hi/lo products x 8 real flops per complex MAC, "
                    "ng_max^2 min(Nv^2, Nc^2) per block; the whole stage's time (splits and block products "
                    "included)",
            "traffic": None, "peak_source": src + " (sustained bf16: timed inside a long step)"}
    ms = st["exchange_kernel"]
    cmac_x = float(dim) * dim * inf["ng0"] / 2
    if prec == 0:
        flops = 8.0 * cmac_x
        out["exchange_kernel"] = {"bound": "alu", "kernel": "init_kernel", "achieved": flops / (ms / 1e3) / 1e12,
                                  "peak": fp32, "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / fp32,
                                  "work": "8 flops per complex MAC of rho_x^H vbar rho_x over the upper triangle",
                                  "traffic": None, "peak_source": "derived FP32 CUDA-core peak", "launches_per_step": 1}
    else:
        flops = 24.0 * cmac_x
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        out["exchange_kernel"] = {
            "bound": "tensor", "kernel": "gram_split_kernel + gram_kernel", "achieved": flops / (ms / 1e3) / 1e12,
            "peak": peak, "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / peak,
            "work": "BF16x3 split-complex flops (24 per complex MAC) of rho_x^H vbar rho_x over the upper triangle; "
                    "the stage's whole time (operand split included)",
            "traffic": None, "peak_source": src + " (sustained bf16: timed inside a long step)", "launches_per_step": 2}
    return out


def _oracle_exchange_rows(spec, s, ik):
    from oracle import geometry as geo, pair as op
    g0 = geo.sphere(spec, (0, 0, 0))
    r = op.rho_corr(spec, ik, ik, list(range(spec.nv)), list(range(spec.nv, spec.nb)), g0, s.gk, s.coef)
    return r.reshape(spec.nv * spec.nc, -1)


def cpu_baseline(spec, s, H32, Hmx, eps32, epsmx, steps_done, budget_s=15.0):
    """The oracle as it stands on the host cores, on a bounded sample of the step, and the errors of the GPU's
    results against it:
      - random upper (k, k') blocks of H (exchange rows, direct pair densities by the correlation sum, K^d
        contraction) within about budget_s, compared with the GPU's FP32 and mixed H blocks (kernel entries,
        i.e. everything but the diagonal transition energies);
      - the oracle's FP64 Haydock recursion (all nsteps) and continued fraction on the system's own H, as the
        GPU's FP32 build produced it, compared with the GPU's eps_2 of both steps.
    The step time is t_block x (upper blocks) + t_exchange_rows x Nk + t_haydock."""
    import numpy as np
    import time as _t
    from oracle import geometry as geo, kernel as ok, pair as op, spectrum as osp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    blocks = geo.upper_blocks(spec)
    rng = np.random.default_rng(0)
    nvc = spec.nv * spec.nc
    vbar = ok.coulomb_bar(spec)
    de = ok.transition_energies(spec, s.energies, spec.delta)
    errs32, errsmx, scale = [], [], 0.0
    t_rows, n_rows, t_dir, n_dir = 0.0, 0, 0.0, 0
    t_start = _t.perf_counter()
    for idx in rng.permutation(len(blocks)):
        ik, ik2 = blocks[idx]
        t0 = _t.perf_counter()
        rx = _oracle_exchange_rows(spec, s, ik)
        rx2 = rx if ik2 == ik else _oracle_exchange_rows(spec, s, ik2)
        t1 = _t.perf_counter()
        iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
        kd = ok.direct_block(spec, rv, rc, ok.w_of_q(spec, s.W, iq))
        t2 = _t.perf_counter()
        t_rows += t1 - t0
        n_rows += 1 if ik2 == ik else 2
        t_dir += t2 - t1
        n_dir += 1
        ref = 2.0 * ok.norm_factor(spec) * (np.conj(rx) * vbar[None, :]) @ rx2.T - kd
        if ik == ik2:
            ref = ref + np.diag(de[ik * nvc:(ik + 1) * nvc])
            ref = 0.5 * (ref + ref.conj().T)
        off = ~np.eye(nvc, dtype=bool) if ik == ik2 else np.ones((nvc, nvc), bool)
        sl = (slice(ik * nvc, (ik + 1) * nvc), slice(ik2 * nvc, (ik2 + 1) * nvc))
        errs32.append(np.abs(H32[sl] - ref)[off])
        errsmx.append(np.abs(Hmx[sl] - ref)[off])
        scale = max(scale, float(np.abs(ref[off]).max()))
        if _t.perf_counter() - t_start > budget_s:
            break
    e32 = np.concatenate(errs32) / scale
    emx = np.concatenate(errsmx) / scale
    # Haydock on the system's own H (the GPU's FP32 build, upcast), all steps of the workload
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    Hd = H32.astype(np.complex128)
    t3 = _t.perf_counter()
    eref, a, b, done = osp.eps2_haydock(spec, Hd, P, s.omega, spec.eta, spec.nsteps)
    t_hay = _t.perf_counter() - t3
    del Hd
    peak = np.abs(eref).max()
    t_step = t_dir / n_dir * len(blocks) + t_rows / n_rows * spec.nkpt + t_hay
    return {"value": spec.dim * spec.dim / t_step, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_dir} random upper (k,k') blocks (direct pair densities by the correlation sum + K^d; "
                      f"{n_rows} exchange-row sets) scaled to {len(blocks)} blocks and {spec.nkpt} row sets, plus "
                      f"the full {spec.nsteps}-step FP64 Haydock and continued fraction on the system's own H "
                      f"(the GPU's FP32 build, upcast to complex128), timed as it ran",
            "est_step_s": t_step, "haydock_s": t_hay,
            "parity": {"blocks": n_dir,
                       "kernel_rel_err_fp32": {"max": float(e32.max()), "mean": float(e32.mean())},
                       "kernel_rel_err_mixed": {"max": float(emx.max()), "mean": float(emx.mean())},
                       "eps2_rel_err_fp32_vs_oracle_haydock": float(np.abs(eps32 - eref).max() / peak),
                       "eps2_rel_err_mixed_vs_oracle_haydock": float(np.abs(epsmx - eref).max() / peak),
                       "oracle_steps_done": int(done), "gpu_steps_done": int(steps_done),
                       "note": "kernel errors relative to the largest sampled kernel entry; eps_2 errors relative "
                               "to the oracle spectrum's peak"}}


def cpu_full_small(runs=3):
    """The oracle's whole step, unsampled, on the tiny bulk cell (fcc 4x4x4 3v3c, dim 576): every pair
    density, the full H (exchange and direct terms) and its Haydock spectrum; the median over runs."""
    import time as _t
    import numpy as np
    from oracle import kernel as ok, pair as op, spectrum as osp
    from synth import config_spec, generate
    spec = config_spec("fcc_4x4x4_3v3c")
    s = generate(spec)
    times = []
    for _ in range(runs):
        t0 = _t.perf_counter()
        H = ok.hamiltonian_full(spec, s.gk, s.coef, s.energies, s.W, spec.delta)
        P = op.dipole(spec, s.gk, s.coef, s.energies)
        osp.eps2_haydock(spec, H, P, s.omega, spec.eta, spec.nsteps)
        times.append(_t.perf_counter() - t0)
    med = float(np.median(times))
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"workload": f"{spec.name}: dim {spec.dim}, {spec.nsteps} Haydock steps, {len(s.omega)} w, whole step",
            "runs": runs, "median_s": med, "value": spec.dim * spec.dim / med, "unit": UNIT, "cores": cores,
            "kind": "oracle"}


def run_reference(args):
    """The oracle alone on the host cores, per step a bounded sample of the same workload: random upper blocks
    (exchange rows, direct pair densities, K^d) within the budget, and Haydock steps of the oracle recursion on a
    dense Hermitian matrix of the workload's dimension (the system's own H needs the full build, which does not
    fit a bounded step), scaled to the full step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import time as _t
    from oracle import geometry as geo, kernel as ok, pair as op, spectrum as osp
    spec, s = make_inputs(args.config)
    blocks = geo.upper_blocks(spec)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rng = np.random.default_rng(0)
    dim = spec.dim
    hay_steps = 4
    m = np.empty((dim, dim), dtype=np.complex128)
    for i in range(0, dim, 2048):
        j = min(i + 2048, dim)
        m[i:j] = rng.standard_normal((j - i, dim)) + 1j * rng.standard_normal((j - i, dim))
    m += m.conj().T
    P = rng.standard_normal(dim) + 0j
    times, ests = [], []
    perm = rng.permutation(len(blocks))
    pos = 0
    for k in range(args.warmup + args.steps):
        t0 = _t.perf_counter()
        t_dir, n_dir, t_rows, n_rows = 0.0, 0, 0.0, 0
        while _t.perf_counter() - t0 < 0.7 * args.cpu_budget:
            ik, ik2 = blocks[perm[pos % len(perm)]]
            pos += 1
            a = _t.perf_counter()
            _oracle_exchange_rows(spec, s, ik)
            b = _t.perf_counter()
            iq, rv, rc = op.direct_rho_block(spec, ik, ik2, s.gk, s.coef)
            ok.direct_block(spec, rv, rc, ok.w_of_q(spec, s.W, iq))
            c = _t.perf_counter()
            t_rows += b - a
            n_rows += 1
            t_dir += c - b
            n_dir += 1
        a = _t.perf_counter()
        osp.haydock(m, P, hay_steps)
        t_hay = (_t.perf_counter() - a) / hay_steps
        est = t_dir / n_dir * len(blocks) + t_rows / n_rows * spec.nkpt + t_hay * spec.nsteps
        if k >= args.warmup:
            times.append(_t.perf_counter() - t0)
            ests.append(est)
    est = statistics.median(ests)
    ng_max = max(len(geo.sphere(spec, tuple(o))) for o in geo.mesh_offsets(spec))
    value = dim * dim / est
    sample = (f"per step: random upper (k,k') blocks for {0.7 * args.cpu_budget:.0f} s (direct pair densities by "
              f"the correlation sum + K^d, exchange rows) and {hay_steps} Haydock steps on a dense Hermitian "
              f"matrix of dim {dim}; scaled to {len(blocks)} blocks, {spec.nkpt} row sets and {spec.nsteps} "
              f"steps; median of {args.steps} steps")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": est * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": dict(workload_config(spec, ng_max), precision="complex128 oracle (CPU), bounded sample per step",
                          parallelism="host cores"),
           "sample_wall_s_per_step": statistics.median(times),
           "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": value},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=HEADLINE)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16x3"], help="precision of --only runs")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip every fcc 8x8x8 and batch measurement")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch of hexagonal sheets")
    ap.add_argument("--no-screening", action="store_true", help="skip the static RPA screening measurement")
    ap.add_argument("--no-coupled", action="store_true", help="skip the BSE with e-h / h-e coupling")
    ap.add_argument("--no-symmetry", action="store_true", help="skip the q-point symmetry measurement")
    ap.add_argument("--no-tddft", action="store_true", help="skip the TDDFT macroscopic dielectric function")
    ap.add_argument("--no-states", action="store_true", help="skip the exciton-state eigensolver")
    ap.add_argument("--only", default="all", choices=["all", "pair", "spectrum", "contract", "exchange"],
                    help="profiling aid: run one stage (pair: realspace + a q chunk of pair densities; "
                         "contract: the direct term of a q chunk; exchange: diagonal + 2 K^x; "
                         "spectrum: Haydock on an H built once before the loop)")
    ap.add_argument("--qchunk", type=int, default=0, help="q points per direct-term chunk (0 = automatic)")
    ap.add_argument("--variant", type=int, default=-1, help="profiling aid for --only pair: pair-kernel variant index")
    ap.add_argument("--nk", type=int, default=0,
                    help="profiling aid for --only: the workload's per-block shape on an nk^3 k mesh")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.only != "all":
        run_stage(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
