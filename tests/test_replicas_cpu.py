"""The multi-GPU form of the benchmark is replicas only: each rank solves its
own chip and only the timing and pair counts are combined.  This covers
that host logic with two gloo ranks on the CPU (no GPU, no NCCL)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 100 + 50 r ms and verified 5000 - r pairs
        t, v = bench.aggregate(100.0 + 50.0 * rank, 5000 - rank, world)
        out[rank] = (t, v)
    finally:
        dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sums_pairs_over_two_gloo_ranks():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (150.0, 9999.0)   # every rank sees the same whole-job figures


def test_single_rank_aggregate_is_identity():
    assert bench.aggregate(12.5, 7, 1) == (12.5, 7.0)


def test_replicas_draw_different_chips():
    w0, w1 = bench.workload(0), bench.workload(1)
    assert w0.chips[0].n == w1.chips[0].n                       # same shape, so the same work per rank
    assert not (w0.chips[0].layer_k == w1.chips[0].layer_k).all()   # but an independent chip


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse_args(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) is None   # returns at once: no oracle work, no output
