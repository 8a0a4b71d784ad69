"""The multi-GPU path of bench.py is replicas only (every rank steps its own copy of
the workload, no collective on the data path): two gloo ranks on the CPU check the
whole-job aggregation -- the slowest rank's time, every rank's node updates."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_max, mlups = bench.whole_job(10.0 + 3.0 * rank, 1000, 50, world, dist)
        out.put((rank, ms_max, mlups))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_updates():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms_max, mlups in res:
        assert ms_max == 13.0
        assert abs(mlups - 2 * 1000 * 50 / (1e3 * 13.0)) < 1e-12


def test_one_rank_is_the_plain_rate():
    import bench

    ms_max, mlups = bench.whole_job(4.0, 2048 * 4096, 200, 1)
    assert ms_max == 4.0 and abs(mlups - 2048 * 4096 * 200 / 4e3) < 1e-9
