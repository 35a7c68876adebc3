"""One system split over two ranks (gloo, CPU, 127.0.0.1): the q partition of the direct term, the row
reduction of H and a row-sharded Haydock recursion, against the single-rank oracle.

Each rank builds its partial H from the oracle's blocks of its own q points (rank 0 adds diag + 2 K^x for
every block), the product's ``reduce_rows`` leaves it its rows of the sum, and the recursion runs on the
row slices with the product's collectives (``allreduce_sum`` for the projections and norms,
``allgather_rows`` for the next vector).  The union of the ranks' q points must be every q exactly once,
the reduced rows must equal the oracle's H, and the sharded recursion's coefficients must equal the
single-rank oracle recursion's.
"""
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _system():
    from synth import SystemSpec, generate
    spec = SystemSpec("split", "fcc", 10.0, 0.0, (3, 3, 3), 2, 2, 2.0, (12, 12, 12), "3d", nsteps=40, nw=200)
    return spec, generate(spec)


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    from oracle import geometry as geo
    from oracle import kernel as ok
    from oracle import pair as op
    from paper_1206_3518_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        spec, s = _system()
        nvc = spec.nv * spec.nc
        kr = geo.mesh_offsets(spec)
        blocks = geo.upper_blocks(spec)
        qof = [geo.fold(spec, kr[a], kr[b])[0] for a, b in blocks]
        ngq = [len(geo.sphere(spec, tuple(kr[q]))) for q in range(spec.nkpt)]
        work = [0.0] * spec.nkpt
        for (a, b), q in zip(blocks, qof):
            work[q] += ngq[q] * ngq[q]
        owner = shard.q_groups(work, world)
        mine = [q for q in range(spec.nkpt) if owner[q] == rank]
        # partial H of this rank (its blocks only; rank 0 also diag + 2 K^x, mirrored)
        H = np.zeros((spec.dim, spec.dim), dtype=np.complex128)
        if rank == 0:
            rx = op.exchange_rho(spec, s.gk, s.coef)
            H += 2.0 * ok.exchange_kernel(spec, rx) + np.diag(ok.transition_energies(spec, s.energies, spec.delta))
        for (a, b), q in zip(blocks, qof):
            if owner[q] != rank:
                continue
            iq, rv, rc = op.direct_rho_block(spec, a, b, s.gk, s.coef)
            kd = ok.direct_block(spec, rv, rc, ok.w_of_q(spec, s.W, iq))
            sl = (slice(a * nvc, (a + 1) * nvc), slice(b * nvc, (b + 1) * nvc))
            blk = H[sl] - kd
            if a == b:
                blk = 0.5 * (blk + blk.conj().T)
            H[sl] = blk
            if a != b:
                H[b * nvc:(b + 1) * nvc, a * nvc:(a + 1) * nvc] = blk.conj().T
        ranges = shard.row_ranges(spec.nkpt, nvc, world)
        r0, r1 = ranges[rank]
        Hloc = shard.reduce_rows(torch.as_tensor(H), ranges, rank).numpy()
        # row-sharded Haydock (classical Gram-Schmidt twice against the whole basis, as the library's)
        P = op.dipole(spec, s.gk, s.coef, s.energies)
        n = spec.nsteps
        v = torch.as_tensor(P / np.linalg.norm(P))
        V = []
        a_co, b_co = np.zeros(n), np.zeros(n)
        for j in range(n):
            V.append(v[r0:r1].numpy().copy())
            w = Hloc @ v.numpy()                                   # local rows of H v
            basis = np.stack(V)                                    # [j+1][local rows]
            h1 = shard.allreduce_sum(torch.as_tensor(np.conj(basis) @ w)).numpy()
            w = w - basis.T @ h1
            h2 = shard.allreduce_sum(torch.as_tensor(np.conj(basis) @ w)).numpy()
            w = w - basis.T @ h2
            a_co[j] = (h1[j] + h2[j]).real
            nrm = np.sqrt(shard.allreduce_sum(torch.as_tensor(np.array([np.vdot(w, w).real]))).numpy()[0])
            if j + 1 < n:
                b_co[j + 1] = nrm
                v = shard.allgather_rows(torch.as_tensor(w / nrm), ranges)
        queue.put((rank, mine, r0, r1, Hloc, a_co, b_co))
    except Exception as e:                       # report instead of leaving the other side waiting
        queue.put((rank, "error", repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_single_system_split_over_two_ranks():
    import torch.multiprocessing as mp
    from oracle import kernel as ok
    from oracle import pair as op
    from oracle import spectrum as osp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted([queue.get(timeout=240) for _ in procs], key=lambda x: x[0])
    assert all(o[1] != "error" for o in out), out
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    spec, s = _system()
    rx = op.exchange_rho(spec, s.gk, s.coef)
    fac = ok.direct_factors(spec, s.gk, s.coef)
    Href = ok.hamiltonian_from_factors(spec, s.energies, spec.delta, rx, fac, s.W)
    P = op.dipole(spec, s.gk, s.coef, s.energies)
    a, b, done, _ = osp.haydock(Href, P, spec.nsteps)
    qs = sorted(out[0][1] + out[1][1])
    assert qs == list(range(spec.nkpt)) and not set(out[0][1]) & set(out[1][1]) and 0 in out[0][1]
    assert out[0][2] == 0 and out[0][3] == out[1][2] and out[1][3] == spec.dim
    for _, _, r0, r1, Hloc, _, _ in out:
        assert np.abs(Hloc - Href[r0:r1]).max() < 1e-12 * np.abs(Href).max()
    assert done == spec.nsteps
    for _, _, _, _, _, a_co, b_co in out:
        assert np.abs(a_co - a).max() < 1e-10 * np.abs(a).max()
        assert np.abs(b_co - b).max() < 1e-10 * np.abs(b).max()


def test_partition_helpers():
    from paper_1206_3518_gb300 import shard
    owner = shard.q_groups([5.0, 1.0, 9.0, 3.0, 3.0, 7.0], 3)
    assert owner[0] == 0 and sorted(set(owner)) == [0, 1, 2]
    load = [sum(w for w, o in zip([5.0, 1.0, 9.0, 3.0, 3.0, 7.0], owner) if o == r) for r in range(3)]
    assert max(load) - min(load) <= 9.0
    assert shard.row_ranges(5, 4, 2) == [(0, 12), (12, 20)]
    assert shard.row_ranges(4, 3, 4) == [(0, 3), (3, 6), (6, 9), (9, 12)]
    assert shard.q_groups([1.0, 2.0], 1) == [0, 0]
