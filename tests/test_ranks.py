"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own model's timings and
texel counts, combine into the whole-job figures (max time, summed texels) on every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
    texels = 1000 * (rank + 1)
    out = bench.combine_ranks(times, texels, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_two_gloo_ranks_combine_max_time_and_summed_texels():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        times, texels = res[r]
        assert times == [11.0, 20.0, 10.0]
        assert texels == 3000.0


def test_single_rank_is_identity():
    import bench
    times, texels = bench.combine_ranks([1.5, 2.5], 42, 1, "cpu")
    assert times == [1.5, 2.5] and texels == 42.0
