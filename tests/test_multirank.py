"""The multi-rank path of bench.py on the CPU: two gloo ranks over 127.0.0.1.

Replicas report the slowest rank's time (all-reduce MAX); the batch of hexagonal sheets is sharded
by balanced dim^2 with no data-path exchange: every rank must compute the same, complete, disjoint
assignment.
"""
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, queue):
    import torch.distributed as dist
    import bench
    from synth import slab_batch_specs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dims = [s.dim for s in slab_batch_specs(0)]
        mine = bench.shard_systems(dims, rank, world)
        everyone = [None] * world
        dist.all_gather_object(everyone, mine)
        mx = bench.max_over_ranks(10.0 + 3.0 * rank, world)
        queue.put((rank, dims, everyone, mx))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    out = [queue.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    dims = out[0][1]
    assert out[0][2] == out[1][2]                       # every rank sees the same assignment
    a, b = out[0][2]
    assert sorted(a + b) == list(range(len(dims))) and not set(a) & set(b)
    la, lb = sum(dims[i] ** 2 for i in a), sum(dims[i] ** 2 for i in b)
    assert abs(la - lb) <= max(d * d for d in dims)     # greedy balance bound
    assert out[0][3] == out[1][3] == 13.0               # slowest rank's time on both


def test_one_rank_is_identity():
    import bench
    assert bench.max_over_ranks(4.5, 1) == 4.5
    assert bench.shard_systems([3, 1, 2], 0, 1) == [0, 1, 2]
