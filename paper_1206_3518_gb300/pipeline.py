"""Chaining of the C-ABI calls into one forward pass of the hot path (A1-A8).

Only buffer allocation (torch) and call order live here; every step runs in
the CUDA library.  ``Forward`` preallocates every buffer for one system so a
timed loop allocates nothing.
"""
from __future__ import annotations

import torch

from . import bse


class Forward:
    """Buffers and call sequence for one system of a plan.

    qchunk: q points per pair-density/direct-term chunk (rho_dir is streamed);
    keep_rho_dir: keep the direct pair densities of every q (needed by the adjoint).
    """

    def __init__(self, plan: bse.Plan, s: int = 0, nsteps: int = 100, nw: int = 1000, qchunk: int | None = None,
                 keep_rho_dir: bool = False, device="cuda"):
        self.plan, self.s = plan, s
        inf = plan.info(s)
        self.info = inf
        self.dim, self.nq, self.ng_max = inf["dim"], inf["nq"], inf["ng_max"]
        self.nsteps = nsteps
        self.tensor_choice = None             # set by autotune.tune(..., with_tensor=True)
        if keep_rho_dir or qchunk is None:
            qchunk = self.nq
        self.qchunk = qchunk
        dev = torch.device(device)
        c64, c128 = torch.complex64, torch.complex128
        self.ws_pair = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_PAIR) // 8, dtype=c64, device=dev)
        self.ws_kernel = torch.empty(max(1, bse.bse_workspace_size(plan, s, bse.BSE_WS_KERNEL, qchunk) // 8),
                                     dtype=c64, device=dev)
        self.ws_spec = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_SPECTRUM, nsteps) // 8 + 1,
                                   dtype=c64, device=dev)
        self.rho_x = torch.zeros(self.dim, self.ng_max, dtype=c64, device=dev)
        self.P = torch.zeros(self.dim, dtype=c128, device=dev)
        self.chunks = [(q, min(q + qchunk, self.nq)) for q in range(0, self.nq, qchunk)]
        nvec = max(bse.bse_rho_dir_count(plan, s, a, b) for a, b in self.chunks)
        self.rho_dir = torch.zeros(nvec, self.ng_max, dtype=c64, device=dev)
        self.H = torch.empty(self.dim, self.dim, dtype=c64, device=dev)
        self.eps2 = torch.zeros(nw, dtype=torch.float64, device=dev)
        self.ab = torch.zeros(2 * nsteps, dtype=torch.float64, device=dev)
        self.steps_done = torch.zeros(1, dtype=torch.int32, device=dev)

    def build(self, coef, energies, W, delta, prec=bse.BSE_PREC_FP32, tensor_pair=None):
        """A1-A6: pair densities, dipole and H (direct term streamed over q chunks).

        tensor_pair: direct pair densities on the tensor cores (BSE_PD_TENSOR); by default with the
        mixed precision where the system has that route, or as the autotuner chose for this system.
        """
        p, s = self.plan, self.s
        if tensor_pair is None:
            tensor_pair = prec == bse.BSE_PREC_BF16X3 and bool(self.info["tensor_pair"])
            if tensor_pair and self.tensor_choice is not None:
                tensor_pair = self.tensor_choice
        fdir = bse.BSE_PD_DIRECT | (bse.BSE_PD_TENSOR if tensor_pair else 0)
        bse.bse_pair_densities(p, s, bse.BSE_PD_REALSPACE | bse.BSE_PD_EXCHANGE, coef, energies, self.rho_x, self.P,
                               None, 0, 0, self.ws_pair)
        bse.bse_build_kernel(p, s, bse.BSE_BK_INIT, self.rho_x, None, 0, 0, None, energies, delta, prec, self.H,
                             self.ws_kernel if prec == bse.BSE_PREC_BF16X3 else None)
        for q0, q1 in self.chunks:
            bse.bse_pair_densities(p, s, fdir, None, None, None, None, self.rho_dir, q0, q1, self.ws_pair)
            bse.bse_build_kernel(p, s, bse.BSE_BK_DIRECT, None, self.rho_dir, q0, q1, W, None, delta, prec, self.H,
                                 self.ws_kernel)
        if self.info["kpoint_symmetry"]:
            bse.bse_build_kernel(p, s, bse.BSE_BK_SYMFILL, None, None, 0, 0, None, None, delta, prec, self.H, None)
        return self.H

    def spectrum(self, omega, eta, nsteps=None):
        """A7-A8 on the current H and P."""
        n = self.nsteps if nsteps is None else nsteps
        bse.bse_spectrum(self.plan, self.s, self.H, self.P, n, omega, eta, self.eps2[: omega.numel()], self.ab,
                         self.steps_done, self.ws_spec)
        return self.eps2[: omega.numel()]


class Coupled:
    """Buffers and call sequence of the BSE with e-h / h-e coupling for the system of ``fwd``.

    The resonant block A is ``fwd.H``; ``build`` needs the real-space wavefunctions and rho_x that
    ``fwd.build`` leaves in place.  The coupling densities are streamed over ``fwd.chunks``.
    """

    def __init__(self, fwd: Forward, nsteps: int | None = None, nw: int | None = None):
        self.fwd = fwd
        plan, s = fwd.plan, fwd.s
        dev = fwd.H.device
        self.nsteps = fwd.nsteps if nsteps is None else nsteps
        nvec = max(bse.bse_rho_cpl_count(plan, s, a, b) for a, b in fwd.chunks)
        self.rho_cpl = torch.zeros(nvec, fwd.ng_max, dtype=torch.complex64, device=dev)
        self.ws = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_COUPLING, fwd.qchunk) // 8 + 1,
                              dtype=torch.complex64, device=dev)
        self.ws_spec = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_COUPLED, self.nsteps) // 8 + 1,
                                   dtype=torch.complex64, device=dev)
        self.Bm = torch.empty(fwd.dim, fwd.dim, dtype=torch.complex64, device=dev)
        self.eps2 = torch.zeros(fwd.eps2.numel() if nw is None else nw, dtype=torch.float64, device=dev)
        self.b = torch.zeros(self.nsteps, dtype=torch.float64, device=dev)
        self.steps_done = torch.zeros(1, dtype=torch.int32, device=dev)

    def build(self, W, prec=bse.BSE_PREC_FP32):
        """Coupling block B = 2 Bx - Bd (exchange from rho_x, direct term streamed over q chunks)."""
        f = self.fwd
        p, s = f.plan, f.s
        bse.bse_build_coupling(p, s, bse.BSE_BC_INIT, f.rho_x, None, 0, 0, None, prec, self.Bm, self.ws)
        for q0, q1 in f.chunks:
            bse.bse_pair_densities(p, s, bse.BSE_PD_COUPLING, None, None, None, None, self.rho_cpl, q0, q1, f.ws_pair)
            bse.bse_build_coupling(p, s, bse.BSE_BC_DIRECT, None, self.rho_cpl, q0, q1, W, prec, self.Bm, self.ws)
        return self.Bm

    def spectrum(self, omega, eta, nsteps=None):
        """eps_2 of H2 = [[A, B], [-conj B, -conj A]] with A = fwd.H."""
        n = self.nsteps if nsteps is None else nsteps
        f = self.fwd
        bse.bse_spectrum_coupled(f.plan, f.s, f.H, self.Bm, f.P, n, omega, eta, self.eps2[: omega.numel()], self.b,
                                 self.steps_done, self.ws_spec)
        return self.eps2[: omega.numel()]


class Batch:
    """Several systems of one plan: per-system builds (q-streamed) and one batched spectrum launch."""

    def __init__(self, plan: bse.Plan, nsteps: int, nw: int, qchunk: int = 64, device="cuda"):
        self.plan, self.nsteps = plan, nsteps
        self.sys = [Forward(plan, s, nsteps=nsteps, nw=nw, qchunk=min(qchunk, plan.info(s)["nq"]), device=device)
                    for s in range(plan.nsys)]

    def build(self, coefs, energies, Ws, deltas, prec=bse.BSE_PREC_FP32):
        for F, c, e, w, dl in zip(self.sys, coefs, energies, Ws, deltas):
            F.build(c, e, w, dl, prec)

    def spectrum(self, omega, eta):
        S = self.sys
        bse.bse_spectrum_batch(self.plan, list(range(len(S))), [F.H for F in S], [F.P for F in S], self.nsteps,
                               omega, eta, [F.eps2[: omega.numel()] for F in S], [F.ab for F in S],
                               [F.steps_done for F in S], [F.ws_spec for F in S])
        return [F.eps2[: omega.numel()] for F in S]
