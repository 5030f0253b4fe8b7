"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks, each with
its own step time, agree on the slowest one, and the job's throughput counts
both ranks' pixels (weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, r, loc = bench._dist_env()
    ms = bench._max_over_ranks(dist, times[rank], torch.device("cpu"))
    dist.barrier()
    q.put((rank, w, r, loc, ms, bench._job_value(w, 1_000_000, ms)))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [2.0, 3.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, r, loc, ms, value in out:
        assert (w, r, loc) == (2, rank, rank)
        assert ms == 3.0
        # 2 ranks x 1 M pixels in 3 ms
        assert value == pytest.approx(2 * 1e6 / 3e-3 / 1e6)


def test_single_rank_is_unchanged():
    import bench

    assert bench._max_over_ranks(None, 1.25, torch.device("cpu")) == 1.25
    assert bench._job_value(1, 16_777_216, 0.28) == pytest.approx(16_777_216 / 0.28e-3 / 1e6)
