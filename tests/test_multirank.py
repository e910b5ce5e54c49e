"""Multi-rank host logic of the benchmark, as two gloo ranks on the CPU.

The path shards by probe position (independent right-hand sides) and its only exchange is the
max-over-ranks time. Checked here with world_size 2: the ranks' position shards are disjoint and
together equal the single-rank list of the same total size, the job time is the slowest rank's,
and the job rate counts every rank's units.
"""
import json
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


def _rank_main(rank, world, port, out_dir):
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n = 4
        z = bench.probe_positions(n, rank, world)
        shards = [None] * world
        dist.all_gather_object(shards, [float(v) for v in z])
        t = bench.max_over_ranks(1.0 + 0.5 * rank, "cpu")
        rate = bench.job_rate(4 * n, world, t)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"shards": shards, "t": t, "rate": rate}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_positions_and_take_max_time(tmp_path):
    import bench
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    full = [float(v) for v in bench.probe_positions(4 * world, 0, 1)]
    for r in res:
        shards = r["shards"]
        assert sum(shards, []) == full                      # contiguous shards, in rank order
        assert not set(shards[0]) & set(shards[1])           # disjoint
        assert r["t"] == 1.5                                 # the slowest rank's time
        assert r["rate"] == pytest.approx(4 * 4 * world / 1.5)


def test_single_rank_helpers_without_process_group():
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.job_rate(10, 1, 2.0) == 5.0
    assert len(bench.probe_positions(3, 0, 1)) == 3
