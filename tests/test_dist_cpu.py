"""Multi-rank bench logic on CPU (gloo, world size 2): each rank gets its own hologram seeds and the
reported time is the maximum over ranks.  No GPU: the replicas exchange nothing on the data path."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    t = bench.max_over_ranks(10.0 + rank, world, torch.device("cpu"))
    bench.barrier(world)
    q.put((rank, t, bench.rank_seeds(rank)))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [11.0, 11.0]  # max over ranks
    assert out[0][2] != out[1][2]  # distinct holograms per rank
