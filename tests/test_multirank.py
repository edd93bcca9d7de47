"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its own replica.

Every GPU of a job advances an independent lattice (the step has no data exchange in this
build), the job time is the slowest rank's and the throughput counts all ranks' nodes."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [12.0, 15.0][rank]  # the second rank is slower
    q.put((rank, bench.reduce_max(ms, dist, "cpu"), bench.job_mlups(1_000_000, 100, world, bench.reduce_max(ms, dist, "cpu"))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == pytest.approx(2 * 1_000_000 * 100 / 15e-3 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.job_mlups(1000, 10, 1, 1.0) == pytest.approx(10.0)
