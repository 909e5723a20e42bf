"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own batch (replicas,
weak scaling).  The whole-job time is the slowest rank's, the work counters are summed; the
reference arm runs on rank 0 only and the other ranks return without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed 10 (r + 1) ms over its own batch of 1000 (r + 1) steps and 10 (r + 1) rays
        t, (steps, rays) = bench.reduce_over_ranks(10.0 * (rank + 1), [1000 * (rank + 1),
                                                                      10 * (rank + 1)], "cpu")
        r, w, _ = bench._env_rank()
        # a rejected clock record on rank 1 alone makes both ranks measure again
        again = bench.any_rank(rank == 1, "cpu")
        out[rank] = (t, steps, rays, r, w, again)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        t, steps, rays, r, w, again = out[rank]
        assert (r, w) == (rank, world)
        assert again
        assert t == 20.0  # the slowest rank
        assert steps == 3000.0 and rays == 30.0  # all ranks' work
    # the bench's value: all ranks' steps over the slowest time
    assert out[0][1] / (out[0][0] / 1e3) == pytest.approx(150000.0)


def _ref_rank(rank, world, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    calls = []
    bench.oracle_sample = lambda *a, **k: calls.append(a) or (1, 1, 1.0, 1)
    import argparse

    bench.run_reference(argparse.Namespace(ref_sample=64, warmup=1, steps=1))
    out[rank] = len(calls)


def test_reference_arm_runs_on_rank_zero_only():
    out = mp.Manager().dict()
    mp.spawn(_ref_rank, args=(2, out), nprocs=2, join=True)
    assert out[0] == 2 and out[1] == 0  # rank 0: warm-up + one step; rank 1: nothing


def test_clock_records_that_reject_a_timing():
    sys.path.insert(0, ROOT)
    import bench

    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert bench.clocks_reject(ok) is None
    assert bench.clocks_reject(dict(ok, sm_mhz=1800.0, reasons=["sw_power_cap"])) is None
    assert bench.clocks_reject(dict(ok, reasons=["sw_power_cap", "hw_slowdown"])) == "hw_slowdown"
    assert bench.clocks_reject(dict(ok, reasons=["sw_thermal_slowdown"])) is not None
    assert bench.clocks_reject(dict(ok, reasons=["hw_thermal_slowdown"])) is not None
    # a clock held low with nothing active: a leftover lock
    assert "no reason" in bench.clocks_reject(dict(ok, sm_mhz=1200.0))
    # no samples at all: nothing to judge by
    assert bench.clocks_reject({"sm_mhz": None, "sm_max_mhz": None,
                                "reasons": ["unsampled"]}) is None
    assert bench.any_rank(True, "cpu") and not bench.any_rank(False, "cpu")
