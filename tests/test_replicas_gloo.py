"""The N > 1 path of bench.py on CPU: two gloo ranks run replicas, the
barrier holds, and the job's throughput uses the slowest rank's time."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ranks = bench.Ranks(world)
    ranks.barrier()
    local = 1.0 + rank           # rank 1 is the slower replica
    slowest = ranks.max(local)
    value = ranks.throughput(npts=1000, steps=4, seconds=slowest)
    out.put((rank, slowest, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_use_the_slowest_time():
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
    for rank, slowest, value in res:
        assert slowest == 2.0
        assert value == pytest.approx(2 * 1000 * 3 * 4 / 2.0 / 1e6)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1)
    r.barrier()
    assert r.max(3.5) == 3.5
    assert r.throughput(100, 2, 1.0) == pytest.approx(100 * 3 * 2 / 1e6)
