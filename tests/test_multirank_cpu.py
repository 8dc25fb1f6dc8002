"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own local time,
agree on the slowest rank's time and on the whole-job throughput (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    m = bench.max_over_ranks(local_ms)
    v = bench.whole_job_gbs(1e9, 4, world, m)
    dist.barrier()
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in res:
        assert m == 150.0
        assert v == pytest.approx(2 * 1e9 * 4 / 0.150 / 1e9)


def test_single_process_is_identity():
    import bench

    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.whole_job_gbs(2e9, 5, 1, 1000.0) == pytest.approx(10.0)
