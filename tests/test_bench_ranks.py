"""Host logic of the benchmark's multi-GPU path (independent replicas, one
process per GPU), run as two gloo ranks on the CPU: the step time is the
maximum over ranks and the job's ms per frame counts every rank's frames."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r measured (r + 1) ms per step
        out = bench.job_timing(float(rank + 1), world, torch.device("cpu"))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_job_timing_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(world):
        t_max, ms_frame, ms_job = res[rank]
        assert t_max == float(world)              # the slowest rank's step time, on every rank
        assert ms_frame == pytest.approx(world / 2.0)
        assert ms_job == pytest.approx(world / 2.0 / world)


def test_job_timing_single_rank():
    import bench
    assert bench.job_timing(3.0, 1, torch.device("cpu")) == (3.0, 1.5, 1.5)
