"""The replica path of bench.py (one problem per rank, no data-path
collective): world_size-2 gloo ranks on the CPU combine their timings into the
slowest rank's time and the iterations of all ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, iters = bench.combine_ranks(dist, 100.0 + 50.0 * rank, 1000 + rank, "cpu")
    q.put((rank, ms, iters))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, iters in out:
        assert ms == 150.0 and iters == 2001
