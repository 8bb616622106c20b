"""The multi-process benchmark path on CPU: two gloo ranks exercise the
barrier, the max-over-ranks timing and the whole-job throughput that
``bench.py`` uses under torchrun (one replica per GPU, no data-path collective)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank              # rank 1 is the slow one
    dist.barrier()
    mx = bench.reduce_max(local_ms, dist, "cpu")
    value = bench.job_throughput(20, world, mx)
    q.put((rank, mx, value, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_timing_and_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, mx, value, env in res:
        assert mx == 150.0
        assert abs(value - 20 * 2 / 0.150) < 1e-9
        assert env == (2, rank, 0)


def test_single_process_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(10, 1, 500.0) == 20.0
