"""The N > 1 path of bench.py (independent replicas, one per GPU) on CPU ranks:
two gloo processes check the max-over-ranks timing and the whole-job value,
and the reference arm's rank != 0 exit.  No GPU is used."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        t = 10.0 + 7.0 * rank                       # rank 1 is the slow one
        t_max = bench.max_over_ranks(dist, t, "cpu")
        value = bench.job_value(world, 100 ** 3, 50 * 4, t_max)
        dist.barrier()
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r\n" % (t_max, value))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [open(tmp_path / ("rank%d.txt" % r)).read().split() for r in range(world)]
    for t_max, value in got:
        assert float(t_max) == 17.0
        assert float(value) == pytest.approx(world * 100 ** 3 * 200 / 17.0)


def test_max_over_ranks_without_a_group_is_the_value():
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:                                        # the arguments the arm reads
        steps, warmup = 1, 0
    assert bench.reference_arm(A, bench.DEFAULT, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
