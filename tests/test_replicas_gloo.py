"""Multi-rank path of the bench on CPU: one process per rank over gloo
(world size 2), as torchrun launches bench.py with --gpus N.  The ray-casting
path needs no exchange between GPUs (replicas only); the only collective is
the timing reduction: whole-job throughput = all ranks' rays / the slowest
rank's time."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    seconds = [2.0, 3.0][rank]                     # rank 1 is the slow one
    rays = 23_592_960 * 10                          # identical replicas
    slowest = bench.barrier_max(seconds, ws)
    rate = bench.aggregate_rate(rays, seconds, ws)
    bench.barrier(ws)
    q.put((rank, slowest, rate))
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, slowest, rate in out:
        assert slowest == 3.0                          # max over ranks
        assert rate == pytest.approx(2 * 23_592_960 * 10 / 3.0)
