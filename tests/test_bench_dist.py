"""The benchmark's multi-rank host logic on CPU: two gloo ranks (world size 2)
run the replica frame split and the max-over-ranks timing exactly as the
GPU ranks do under torchrun, with no GPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        frames = bench.rank_frames(rank, world, 100, 10)
        local_ms = 10.0 + 4.0 * rank  # rank 1 is the slower one
        slowest = bench.max_over_ranks(local_ms, world)
        out[rank] = (frames, slowest, bench.whole_job_ms(slowest, 10, world))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_frames_and_take_the_slowest():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    f0, f1 = res[0][0], res[1][0]
    assert not set(f0) & set(f1) and len(set(f0) | set(f1)) == 20
    for r in range(world):
        frames, slowest, (per_query, per_step) = res[r]
        assert slowest == 14.0  # every rank sees the slowest rank's total
        assert per_query == pytest.approx(14.0 / 20) and per_step == pytest.approx(14.0 / 10)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.rank_frames(0, 1, 5, 7) == [0, 1, 2, 3, 4, 0, 1]
