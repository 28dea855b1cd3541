"""Multi-rank host logic of the benchmark on CPU (two gloo ranks).

One process per GPU runs independent replicas of the solve; the job's rate
is the units every rank processed over the slowest rank's time.  These tests
run that reduction with the gloo backend on the host, no GPU involved."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dev = torch.device("cpu")
        ms = [400.0, 250.0][rank]             # rank 0 is the slower one
        units = [1.0e6, 1.2e6][rank]          # replicas may process different counts
        out[rank] = (bench.reduce_over_ranks(ms, world, dev, "max"),
                     bench.reduce_over_ranks(units, world, dev, "sum"),
                     bench.whole_job_rate(units, ms, world, dev))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_uses_the_slowest_rank_over_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
        assert all(p.exitcode == 0 for p in procs)
        res = dict(out)
    for r in range(world):
        slowest, total, rate = res[r]
        assert slowest == 400.0
        assert total == pytest.approx(2.2e6)
        assert rate == pytest.approx(2.2e6 / 0.4)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.5, 1, torch.device("cpu"), "max") == 3.5
    assert bench.whole_job_rate(1000.0, 500.0, 1, torch.device("cpu")) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    """Under several ranks the oracle arm is timed by rank 0 alone; the others
    leave at once without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1) is None
    assert capsys.readouterr().out == ""
