"""The multi-GPU form of the benchmark is replicas (every rank solves its own
instance; nothing is exchanged on the data path).  Its host logic -- the rank
environment and the whole-job aggregation (units summed over ranks, the
slowest rank's time) -- runs here on CPU with two gloo ranks."""
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


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    ws, r, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    ctx = {"torch": torch, "ws": ws, "dist": dist}
    units = 1000.0 * (r + 1)           # rank r did (r + 1) thousand updates ...
    t_total = 0.5 + 0.25 * r           # ... in 0.5 + 0.25 r seconds
    q.put((r, ws, local) + bench.aggregate(ctx, units, t_total))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r, (rank, ws, local, units, t) in enumerate(out):
        assert (rank, ws, local) == (r, world, r)
        assert units == 3000.0              # summed over ranks
        assert t == 0.75                    # the slowest rank


def test_single_rank_is_identity():
    import bench
    ctx = {"torch": torch, "ws": 1, "dist": None}
    assert bench.aggregate(ctx, 123.0, 4.5) == (123.0, 4.5)
