"""Two ranks driving the library, summed once at the end (-m gpu).

Two processes (gloo on CPU tensors for the one collective) each build the
grid and the k-d tree of the same weighted catalogue on the GPU, count only
their block shard (pc_opts.shard_index / shard_count) through pc_count_auto
and pc_count_tree, and sum the int64 counts and binary64 weighted sums with
shard.sum_histograms -- Sect. 4.3's split with no communication while
counting and one gather at the end.  The sums must equal the oracle's
histogram: counts bit-exact, weighted sums within 1e-10 relative.  The two
ranks share the one GPU; their kernels never wait on each other.
"""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu

L = 300.0
EDGES = np.linspace(0.0, 60.0, 13)


def _catalogue():
    import synth
    x = synth.mixed_box(100_000, L, 0.5, 10.0, 5.0, synth.SEED_BASE + 650)
    w = synth.lognormal_weights(x.shape[0], 0.3, synth.SEED_BASE + 651)
    return x, w


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    try:
        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        import paper_2301_12557_gb300 as P
        from paper_2301_12557_gb300 import shard
        torch.cuda.set_device(0)
        x, w = _catalogue()
        xd, wd = torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda()
        bins = P.Bins("s", "z", EDGES)
        box = P.make_box(L, True)
        out = {}
        opts = shard.shard_opts(P.make_opts("f32", 0.0, 2), rank, world)
        g = P.pc_build_grid(xd, wd, box=box, r_max=bins.r_max, opts=opts)
        try:
            c, wc, st = P.pc_count_auto(g, bins, opts, weighted=True)
        finally:
            g.free()
        out["grid"] = (shard.sum_histograms(c), shard.sum_histograms(wc), int(st.wsum))
        topts = shard.shard_opts(P.make_opts("f32", 0.0, 2), rank, world)
        t = P.pc_build_tree(xd, wd, box=box)
        try:
            c, wc, _ = P.pc_count_tree(t, None, bins, topts, weighted=True)
        finally:
            t.free()
        out["tree"] = (shard.sum_histograms(c), shard.sum_histograms(wc), 0)
        part = int(c.sum())
        parts = shard.sum_histograms(np.array([part, 1], dtype=np.int64))
        if rank == 0:
            q.put(("ok", out, part, parts.tolist()))
        dist.barrier()
        dist.destroy_process_group()
    except Exception as e:  # pragma: no cover
        q.put(("error", repr(e), None, None))


def test_two_ranks_shard_the_library_and_sum_once():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    import paper_2301_12557_gb300 as P
    P.build()
    oracle.build()
    x, w = _catalogue()
    want, wwant = oracle.count(x, w1=w, box=L, periodic=True, edges_a=EDGES, method="grid")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    status, out, part, parts = q.get(timeout=600)
    for p in procs:
        p.join(timeout=600)
    assert status == "ok", out
    assert all(p.exitcode == 0 for p in procs)
    # each rank did part of the work, and the parts add up
    assert parts[1] == 2 and 0 < part < parts[0] == int(want.sum())
    for path in ("grid", "tree"):
        c, wc, wsum = out[path]
        assert np.array_equal(c, want), path
        rel = np.abs(wc - wwant) / np.maximum(np.abs(wwant), 1e-300)
        assert rel.max() <= 1e-10, (path, rel.max())
    assert out["grid"][2] == 2      # the integer weight-product path ran
