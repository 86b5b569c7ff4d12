"""The multi-rank path of the benchmark on CPU: two gloo ranks (replicas), max-over-ranks
timing and the whole-job aggregate. The projector itself needs no exchange between GPUs,
so this is the only N > 1 logic there is."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(10.0 * (rank + 1), torch.device("cpu"))
    val = bench.aggregate_gvv_s(1e9, 2, ms, world)
    dist.destroy_process_group()
    q.put((rank, ms, val))


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    # 2 replicas x 1e9 units x 2 steps in 20 ms
    assert out[0][2] == pytest.approx(2 * 1e9 * 2 / 0.020 / 1e9)


def test_single_process_is_unchanged():
    import torch

    import bench

    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
