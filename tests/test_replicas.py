"""The multi-GPU path is replicas only (independent frames per rank, no data-path collective):
the host logic that bench.py runs on every rank, on CPU with the gloo backend and two ranks.
The slowest rank's time sets the whole job's throughput, every rank sees the same figure, the
ranks render distinct realisations, and the reference arm runs on rank 0 alone."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 17.0][rank]  # rank 1 is slower
    worst = bench.max_over_ranks(ms, world, "cpu")
    rate = bench.whole_job_rate(1000, world, worst * 1e-3)
    out[rank] = (worst, rate, bench.replica_seed(7, rank), bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world = 2
    with mp.get_context("spawn").Manager() as m:  # no fork from a multi-threaded test process
        out = m.dict()
        mp.start_processes(_rank, args=(world, free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        worst, rate, seed, env = res[r]
        assert worst == 17.0
        assert rate == pytest.approx(1000 * world / 17.0e-3)
        assert env == (r, world, r)
    assert res[0][2] != res[1][2]


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.replica_seed(5, 0) == 5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    # rank 1 returns before touching the oracle or the workload
    assert bench.run_reference(None, None) is None
