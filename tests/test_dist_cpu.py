"""Replica scaling logic of bench.py on CPU with the gloo backend (world size 2):
the job time is the slowest rank's, the throughput counts every replica."""
from __future__ import annotations

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


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank            # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (ms_max, bench.whole_job_throughput(1000, 2, world, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput_gloo():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms_max, thr = out[r]
        assert ms_max == 150.0
        assert thr == pytest.approx(1000 * 2 * 2 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.whole_job_throughput(10, 3, 1, 1000.0) == pytest.approx(30.0)


def test_ensemble_members_shard_over_ranks():
    """Every member on exactly one rank, shards differing by at most one."""
    import bench
    for world in (1, 2, 3, 8):
        shards = [bench.shard_members(256, r, world) for r in range(world)]
        flat = sorted(q for sh in shards for q in sh)
        assert flat == list(range(256))
        sizes = [len(sh) for sh in shards]
        assert max(sizes) - min(sizes) <= 1


def test_fp64_colimit_of_the_roofline():
    """The bench's FP64 figure: flops per cell x cells / launch time against
    the measured FP64 peak (the forward sweep at 0.436 ms on 1.122 M cells
    runs 72 flop/cell = 0.185 TFLOP/s, 0.156 of 1.19)."""
    import bench
    r = bench.fp64_colimit("ilu_fwd_sweep", 1_122_000, 0.436e-3)
    assert r["flops_per_cell"] == 72
    assert r["achieved_tflops"] == pytest.approx(0.1853, abs=1e-4)
    assert r["frac"] == pytest.approx(0.1853 / 1.19, abs=1e-4)
    assert bench.fp64_colimit("cpr_apply", 1000, 1e-3) is None
    assert bench.fp64_colimit("spmv_wells", 1000, 0.0) is None
    for k in bench.ALGO_BYTES_PER_CELL:
        assert k in bench.ALGO_FP64_FLOPS_PER_CELL
