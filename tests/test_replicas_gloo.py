"""The multi-process path of the bench on CPU (gloo, world size 2).  The method needs
no exchange between GPUs here: each rank runs an independent replica, and the bench
only reduces the step time (max over ranks) and reports the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.replica_time(times[rank], ws, "cpu")
    rate = bench.aggregate_rate(1000, ws, ms)
    # a failed replica passes inf: every rank sees it
    failed = bench.replica_time(float("inf") if rank == 1 else 1.0, ws, "cpu")
    out.put((rank, ms, rate, failed))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_time_is_max_over_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, [2.0, 5.0], q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate, failed in res:
        assert ms == 5.0
        assert rate == pytest.approx(2 * 1000 / 5e-3)
        assert failed == float("inf")


def test_single_rank_passthrough():
    import bench
    assert bench.replica_time(3.0, 1, "cpu") == 3.0
    assert bench.aggregate_rate(10, 1, 2.0) == pytest.approx(5000.0)
