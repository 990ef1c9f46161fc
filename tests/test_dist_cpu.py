"""The multi-rank timing path of bench.py on two gloo ranks (CPU): every
rank reports its own time, all of them get the slowest one."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                      # this rank's own time
    got = bench.max_over_ranks(dist, torch, ms, device="cpu")
    frames = world * bench.FRAMES * 3           # value = all ranks' frames / slowest time
    q.put((rank, got, frames / (got / 1e3)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_aggregate_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 64 * 3 / 0.015)
