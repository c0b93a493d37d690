"""Multi-rank host logic on CPU (gloo, world size 2): each rank counts its
shard of i-points against the whole catalogue, the histograms are summed with
one collective, and the sum must equal the unsharded count -- the gather-at-
the-end design of Sect. 4.3.  Counting here uses the CPU oracle, so no GPU is
needed; the GPU kernels' own sharding is covered by
test_gpu_parity.py::test_block_shards_sum_to_the_full_count."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import oracle
        import synth
        from paper_2301_12557_gb300 import shard
        L = 80.0
        x = synth.neyman_scott(1500, 150, 10.0, 2.0, L, 501)
        ea = np.linspace(0.0, 16.0, 9)
        mu = np.linspace(0.0, 1.0, 6)
        mine = shard.shard_units(x.shape[0], rank, world)
        part, _ = oracle.count(x[mine], x, box=L, periodic=True, mode="smu", edges_a=ea,
                               edges_b=mu, threads=2)
        total = shard.sum_histograms(part)
        t = torch.tensor([float(rank + 1)], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)     # the bench's max-over-ranks timing
        if rank == 0:
            auto, _ = oracle.count(x, box=L, periodic=True, mode="smu", edges_a=ea, edges_b=mu,
                                   threads=2)
            want = 2 * auto
            want[0] += x.shape[0]                     # self pairs land in bin 0
            q.put((bool(np.array_equal(total, want)), float(t.item())))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # pragma: no cover
        q.put(("error", repr(e)))


def test_two_rank_shards_sum_to_the_full_count():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=240)
    for p in procs:
        p.join(timeout=240)
    assert res == (True, 2.0), res
    assert all(p.exitcode == 0 for p in procs)


def _max_worker(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import bench
        v = bench.max_over_ranks(10.0 * (rank + 1), dist, torch.device("cpu"))
        q.put((rank, v))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # pragma: no cover
        q.put(("error", repr(e)))


def test_bench_max_over_ranks():
    """The benchmark's max-over-ranks reduction (its timing rule) on two gloo
    ranks, and its one-process form."""
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=240)
    assert res == [(0, 20.0), (1, 20.0)], res


def test_shard_units_partition():
    from paper_2301_12557_gb300 import shard
    for n in (0, 1, 7, 256):
        for world in (1, 2, 3, 8):
            seen = sorted(u for r in range(world) for u in shard.shard_units(n, r, world))
            assert seen == list(range(n))
