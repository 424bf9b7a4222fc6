"""The benchmark's multi-rank host logic on CPU: two gloo ranks shard the
frames of one trajectory, take the slowest rank's time and compute the
whole-job throughput; the reference arm does its work on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, frames, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import torch
        import torch.distributed as dist
        dist.init_process_group("gloo", rank=rank, world_size=world)
        fids = bench.frame_shard(rank, world, frames)
        shards = [None] * world
        dist.all_gather_object(shards, fids)
        own_ms = 100.0 + 37.5 * rank           # each rank's own timed total
        job_ms = bench.max_over_ranks(own_ms, torch.device("cpu"))
        value = bench.job_value(frames, 3, world, job_ms)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, shards, own_ms, job_ms, value))
    except Exception as e:   # reported to the parent, which fails the test
        q.put((rank, repr(e), None, None, None))


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    frames = 5
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, frames, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        rank, shards, own, job, value = q.get(timeout=120)
        assert not isinstance(shards, str), shards
        out[rank] = (shards, own, job, value)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(o[1] for o in out.values())
    for rank, (shards, own, job, value) in out.items():
        flat = [f for s in shards for f in s]
        assert sorted(flat) == list(range(world * frames))       # every frame once
        assert len(set(flat)) == len(flat)
        assert shards[rank] == bench.frame_shard(rank, world, frames)
        assert job == slowest                                      # max over ranks on every rank
        assert value == pytest.approx(world * frames * 3 / (slowest / 1000.0))


def test_single_rank_helpers():
    assert bench.frame_shard(0, 1, 4) == [0, 1, 2, 3]
    assert bench.frame_shard(2, 4, 3) == [6, 7, 8]
    assert bench.frame_shard(0, 1, 0) == []
    with pytest.raises(ValueError):
        bench.frame_shard(2, 2, 4)
    import torch
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5   # no process group: the value itself
    assert bench.job_value(64, 10, 1, 500.0) == pytest.approx(1280.0)


def test_reference_arm_other_ranks_do_nothing(monkeypatch):
    """Under torchrun only rank 0 runs the oracle; the others exit 0 at once."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    def boom(*a, **k):
        raise AssertionError("rank 1 built the workload")

    monkeypatch.setattr(bench, "workload", boom)

    class A:
        frames, small, cpu_rays, warmup, steps, gpus = 64, False, 8192, 3, 2, 2

    assert bench.run_reference(A()) == 0
