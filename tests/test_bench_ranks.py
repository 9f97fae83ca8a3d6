"""bench.py's whole-job figures for N replicas (max time over ranks, summed work), on CPU with
world-size-2 gloo process groups — the host-side logic of `bench.py --gpus N` under torchrun."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 20.0 - rank]        # rank 1 is slower in the first figure, rank 0 in the second
    work = [100.0 * (rank + 1), 7.0]
    q.put((rank, bench.reduce_over_ranks(times, work, device="cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_world_two():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        mx, sm = got[r]
        assert mx == [11.0, 20.0] and sm == [300.0, 14.0]


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks([3.0], [5.0], device="cpu") == ([3.0], [5.0])
