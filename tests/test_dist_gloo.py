"""The benchmark's multi-rank path on CPU: two gloo ranks reduce their step times with a MAX and
aggregate whole-job throughput (weak scaling: each rank computes its own waveforms)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank
    m = bench.dist_max(ms_local)
    dist.barrier()
    q.put((rank, m, bench.aggregate_value(m, world)))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_value():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 15.0
        assert abs(v - 2 * 1000.0 / 15.0) < 1e-9


def test_single_process_is_identity():
    import bench
    assert bench.dist_max(3.5) == 3.5
    assert bench.aggregate_value(2.0, 1) == 500.0
