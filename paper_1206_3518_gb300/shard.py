"""Splitting one system over several GPUs (one process per GPU): partition and collective schedule.

The direct term (Eq. W_SS) is a sum of independent (k, k') blocks grouped by q = k' - k, and the
Haydock recursion needs only products H x and inner products.  The split is therefore:

1. Build.  Rank 0 owns q = 0 (the diagonal blocks) and writes diag + 2 K^x with the mirrored lower
   triangle (bse_build_kernel INIT | MIRROR); every other rank starts from H = 0.  The q points are
   assigned by ``q_groups`` (balanced by the direct-term work of each q, the same on every rank); each
   rank computes the pair densities and K^d of its own q points only (bse_pair_densities DIRECT +
   bse_build_kernel DIRECT over its q list), which subtracts the blocks and writes their mirrors.  Every
   step is linear in the blocks, so sum_r H_r is the single-GPU H exactly.  W is needed only for the
   rank's own q points, u and rho_x are replicated.
2. Exchange.  ``reduce_rows`` sums the partial H over ranks and leaves each rank its row range
   (``row_ranges``: whole k blocks, balanced rows) - one reduce-scatter of dim^2 complex64.
3. Spectrum.  Each Haydock step multiplies the local rows by the full Lanczos vector, reduces the
   projections (a_j and the 2 x (j + 1) reorthogonalisation coefficients) and the norm b_{j+1} over ranks
   (``allreduce_sum``), and gathers the next vector from its row slices (``allgather_rows``): one
   all-gather of dim complex128 and three small all-reduces per step.

This module holds only the partition and the collectives (torch.distributed, any backend); the per-rank
arithmetic is the library's.  No tensor-memory access crosses GPUs.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def q_groups(work: Sequence[float], world: int) -> List[int]:
    """Owner rank of every q: q = 0 to rank 0, then the remaining q by descending work, each to the least
    loaded rank (ties: lower rank, then lower q).  Deterministic, so every rank computes the same owners."""
    nq = len(work)
    owner = [0] * nq
    load = [0.0] * world
    if nq == 0:
        return owner
    load[0] += float(work[0])
    for q in sorted(range(1, nq), key=lambda q: (-float(work[q]), q)):
        r = min(range(world), key=lambda r: (load[r], r))
        owner[q] = r
        load[r] += float(work[q])
    return owner


def direct_work(plan, s: int = 0) -> List[float]:
    """Direct-term work of each q of system s: blocks x (NG(q)^2 for W.R + NG(q) |S(k')| per band product for
    the pair densities), from the plan's tables (host or device plan)."""
    from . import bse
    inf = plan.info(s)
    npw = [len(bse.bse_gvectors(plan, s, k, 0)) for k in range(inf["nkpt"])]
    out = []
    for q in range(inf["nq"]):
        ng = len(bse.bse_gvectors(plan, s, q, 1))
        blk, _ = bse.bse_pair_blocks(plan, s, q)
        out.append(float(sum(ng * ng + ng * npw[int(k2)] for _, k2 in blk)))
    return out


def row_ranges(nkpt: int, nvc: int, world: int) -> List[Tuple[int, int]]:
    """Row range [r0, r1) of H per rank: contiguous whole k blocks (nvc rows each), sizes differing by at
    most one block."""
    base, extra = divmod(nkpt, world)
    out, k = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k * nvc, (k + n) * nvc))
        k += n
    return out


def reduce_rows(H, ranges, rank: int, group=None):
    """Rows ranges[rank] of sum over ranks of H (every rank passes its full-size partial H).  NCCL: one
    reduce-scatter; other backends: all-reduce, then the slice."""
    import torch
    import torch.distributed as dist
    r0, r1 = ranges[rank]
    if dist.get_backend(group) == "nccl" and all(b - a == ranges[0][1] - ranges[0][0] for a, b in ranges):
        out = torch.empty((r1 - r0,) + tuple(H.shape[1:]), dtype=H.dtype, device=H.device)
        dist.reduce_scatter_tensor(out, H.contiguous(), group=group)
        return out
    t = H.clone()
    dist.all_reduce(t, group=group)
    return t[r0:r1].clone()


def allgather_rows(x_local, ranges, group=None):
    """The full vector from every rank's row slice (slices in rank order, sizes from ranges).  Slices are
    padded to the largest one for the all-gather (equal sizes on every backend), then trimmed."""
    import torch
    import torch.distributed as dist
    m = max(b - a for a, b in ranges)
    tail = tuple(x_local.shape[1:])
    send = torch.zeros((m,) + tail, dtype=x_local.dtype, device=x_local.device)
    send[: x_local.shape[0]] = x_local
    parts = [torch.empty((m,) + tail, dtype=x_local.dtype, device=x_local.device) for _ in ranges]
    dist.all_gather(parts, send, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, ranges)], dim=0)


def allreduce_sum(t, group=None):
    """In-place sum over ranks (projections, norms)."""
    import torch.distributed as dist
    dist.all_reduce(t, group=group)
    return t
