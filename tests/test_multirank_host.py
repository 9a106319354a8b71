"""Multi-GPU runs are independent replicas (one QP per rank, no data-path collective): the
bench's whole-job value is all ranks' solves over the slowest rank's time.  This exercises
that aggregation with two gloo ranks on the CPU."""
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import os
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0, 90.0][rank]
    mx = bench.max_over_ranks(local_ms, device="cpu")
    q.put((rank, mx, bench.replica_rate(5, world, mx)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_rate_over_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max([120.0, 150.0, 90.0][:world])
    for rank, mx, val in res:
        assert mx == slowest
        assert val == pytest.approx(5 * world / (slowest / 1000.0))


def test_single_process_identity():
    import bench
    assert bench.max_over_ranks(12.5, device="cpu") == 12.5
    assert bench.replica_rate(4, 1, 500.0) == pytest.approx(8.0)
