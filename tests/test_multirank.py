"""The N > 1 benchmark path on CPU: world_size-2 gloo ranks (replicas only,
no exchange between GPUs on the data path). Each rank times its own replica;
rank 0 reports all ranks' work over the slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seconds = [2.0, 3.0][rank]                      # rank 1 is the slow one
    t = bench.max_over_ranks(seconds, dist, device="cpu")
    value = bench.whole_job_rate(5, world, t)        # 5 solves per rank
    dist.barrier()
    q.put((rank, t, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_time_and_whole_job_rate():
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
    for rank, t, value in res:
        assert t == 3.0                    # the slowest rank's time on every rank
        assert value == pytest.approx(10 / 3.0)


def test_single_process_passthrough():
    import bench
    assert bench.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(4, 1, 2.0) == 2.0
