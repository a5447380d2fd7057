"""Multi-rank bench aggregation on CPU: two gloo ranks, each with its own
step time, agree on the slowest rank's time and on the whole-job rate."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms, e2e_s = bench.rank_max([100.0 + 50.0 * rank, 0.2 + 0.1 * (1 - rank)], dist, "cpu")
    q.put((rank, step_ms, e2e_s, bench.pairs_per_second(step_ms, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, step_ms, e2e_s, rate in out:
        assert step_ms == 150.0 and abs(e2e_s - 0.3) < 1e-12
        assert rate == 2 * 1000.0 / 150.0


def test_single_rank_is_identity():
    import bench
    assert bench.rank_max([3.0, 4.0], None, "cpu") == [3.0, 4.0]
    assert bench.pairs_per_second(500.0, 1) == 2.0
