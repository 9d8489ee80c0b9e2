"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own replica time.

Each rank of a multi-GPU run processes its own copy of the workload (independent problems,
no data-path collective); the job's step time is the slowest rank's and the reported value
is all ranks' elements over that time.  These tests run that aggregation with world size 2
over gloo, with a rank that is deliberately slower.
"""
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


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_rank = 10.0 + 5.0 * rank          # rank 1 is slower
    ms = bench.max_over_ranks(ms_rank, world, "cpu")
    value = bench.weak_scaling_value(1000, world, ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{ms} {value}\n")
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_scaling_value_with_gloo(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    results = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(world)]
    for ms, value in results:
        assert float(ms) == pytest.approx(15.0)            # the slowest rank's time on every rank
        assert float(value) == pytest.approx(2 * 1000 / 15e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.weak_scaling_value(2_097_152, 1, 86.0) == pytest.approx(2_097_152 / 0.086)
    assert not dist.is_initialized()
