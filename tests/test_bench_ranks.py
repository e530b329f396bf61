"""The multi-GPU path is N independent replicas; the benchmark combines the
ranks' numbers with two host collectives (max of elapsed time, sum of flops).
Checked here with world_size 2 on the gloo backend (CPU)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    elapsed, flops = bench.combine_ranks(dist, 1.0 + rank, 10.0 * (rank + 1), "cpu")
    out[rank] = (elapsed, flops)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (2.0, 30.0) and out[1] == (2.0, 30.0)


def test_combine_ranks_single():
    import bench
    assert bench.combine_ranks(None, 3.0, 7.0, "cpu") == (3.0, 7.0)
