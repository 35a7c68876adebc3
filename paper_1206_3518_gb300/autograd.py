"""eps_2 as a differentiable function of (Delta, W, rho_x, rho_dir) behind torch.autograd.

Forward: H = diag(e_c + Delta - e_v) + 2K^x - K^d (bse_build_kernel, all q) and the Haydock
spectrum (bse_spectrum).  Backward: bse_spectrum_backward (Lanczos recomputed, Krylov
resolvent, hand-written chain to Delta, W and the pair densities).  Marshalling only; every
step runs in the CUDA library.
"""
from __future__ import annotations

import torch

from . import bse


class Eps2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta, W, rho_x, rho_dir, plan, s, energies, P, omega, eta, nsteps):
        inf = plan.info(s)
        dim, nq = inf["dim"], inf["nq"]
        dev = W.device
        H = torch.empty(dim, dim, dtype=torch.complex64, device=dev)
        ws_k = torch.empty(max(1, bse.bse_workspace_size(plan, s, bse.BSE_WS_KERNEL, nq) // 8), dtype=torch.complex64,
                           device=dev)
        d = float(delta.item())
        bse.bse_build_kernel(plan, s, bse.BSE_BK_INIT | bse.BSE_BK_DIRECT, rho_x, rho_dir, 0, nq, W, energies, d,
                             bse.BSE_PREC_FP32, H, ws_k)
        ws_s = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_SPECTRUM, nsteps) // 8 + 1,
                           dtype=torch.complex64, device=dev)
        eps2 = torch.empty(omega.numel(), dtype=torch.float64, device=dev)
        ab = torch.empty(2 * nsteps, dtype=torch.float64, device=dev)
        done = torch.empty(1, dtype=torch.int32, device=dev)
        bse.bse_spectrum(plan, s, H, P, nsteps, omega, eta, eps2, ab, done, ws_s)
        ctx.save_for_backward(W, rho_x, rho_dir, P, omega, H)
        ctx.cfg = (plan, s, eta, nsteps)
        return eps2

    @staticmethod
    def backward(ctx, g):
        W, rho_x, rho_dir, P, omega, H = ctx.saved_tensors
        plan, s, eta, nsteps = ctx.cfg
        dev = W.device
        ws = torch.empty(bse.bse_workspace_size(plan, s, bse.BSE_WS_BACKWARD, nsteps) // 8 + 1, dtype=torch.complex64,
                         device=dev)
        dd = torch.zeros(1, dtype=torch.float64, device=dev)
        dW = torch.zeros_like(W)
        drx = torch.zeros_like(rho_x)
        drd = torch.zeros_like(rho_dir)
        bse.bse_spectrum_backward(plan, s, H, P, nsteps, omega, eta, g.contiguous().to(torch.float64), rho_x, rho_dir,
                                  W, dd, None, drx, drd, dW, ws)
        return dd.reshape(()), dW, drx, drd, None, None, None, None, None, None, None


def eps2(delta, W, rho_x, rho_dir, plan, s, energies, P, omega, eta, nsteps):
    """eps_2(omega) with gradients for delta (0-d float64 tensor), W, rho_x and rho_dir (complex64)."""
    return Eps2.apply(delta, W, rho_x, rho_dir, plan, s, energies, P, omega, eta, nsteps)
