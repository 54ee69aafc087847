"""Multi-rank host logic on CPU (gloo, world size 2): the sharding of
batched fields over ranks (longest first, every field on exactly one rank,
balanced loads), the partition of the serving request stream over ranks
(every request on exactly one rank, bytes balanced), and the timing
reduction the benchmark applies (barrier, maximum over ranks), run as two
processes with a 127.0.0.1 rendezvous."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_2010_05872_gb300 import fields as F  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    shapes, _ = F.batched_shapes()
    weights = [float(a * b * c) for a, b, c in shapes]
    mine = bench.lpt_assign(weights, world)[rank]
    # Every rank computes the same assignment; gather what each rank takes.
    got = [None] * world
    dist.all_gather_object(got, mine)
    # The benchmark's reduction: the slowest rank's time.
    t = torch.tensor([10.0 + rank], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    load = sum(weights[i] for i in mine)
    loads = [None] * world
    dist.all_gather_object(loads, load)
    if rank == 0:
        out.put((got, t.item(), loads, len(shapes)))
    dist.destroy_process_group()


def test_batched_sharding_and_max_timing_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax, loads, n = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    flat = sorted(i for part in got for i in part)
    assert flat == list(range(n))                      # each field exactly once
    assert tmax == 11.0                                # the maximum over ranks
    assert max(loads) <= 1.05 * min(loads)             # longest-first balance


def _serving_worker(rank, world, port, out):
    import numpy as np
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(F.SEED_SERVING)
    sizes = [int(v) for v in rng.choice([4 << 20, 16 << 20, 64 << 20, 540 << 20], size=500)]
    assign = bench.serving_assign(sizes, world)
    mine = [k for k, r in enumerate(assign) if r == rank]
    got = [None] * world
    dist.all_gather_object(got, (mine, assign))
    if rank == 0:
        out.put((got, sizes))
    dist.destroy_process_group()


def test_serving_partition_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_serving_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, sizes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (mine0, a0), (mine1, a1) = got
    assert a0 == a1                                    # the same partition on every rank
    assert sorted(mine0 + mine1) == list(range(len(sizes)))
    assert not set(mine0) & set(mine1)
    b0, b1 = sum(sizes[k] for k in mine0), sum(sizes[k] for k in mine1)
    # Online greedy: the loads differ by at most the largest request.
    assert abs(b0 - b1) <= max(sizes)
