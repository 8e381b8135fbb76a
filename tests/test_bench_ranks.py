"""CPU: the multi-rank path of bench.py (independent replicas, one per rank) on two gloo ranks.

The whole-job value takes the slowest rank's time and the points of all ranks; this runs the
same helper the bench uses under torchrun, over a real two-process group on 127.0.0.1.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, pts = bench.combine_ranks(10.0 + 5.0 * rank, 1e9 * (rank + 1), dist)
    out[rank] = (ms, pts)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, pts = res[rank]
        assert ms == 15.0                 # the slowest rank
        assert pts == 3e9                 # all ranks' points


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(7.0, 5.0, None) == (7.0, 5.0)


def test_roofline_traffic_only_for_the_captured_kernel_family():
    # The bench reports an ncu DRAM figure only while the autotuner kept the kernel family that
    # was captured for that pass (or ran without the autotuner).
    sys.path.insert(0, ROOT)
    import bench
    table = {"rows_pass2": (1.0e9, 2, "rows_one_block")}
    assert bench._traffic(table, "rows_pass2", None) == 1.0e9
    assert bench._traffic(table, "rows_pass2", [{"pass": 2, "chosen": "rows_one_block"}]) == 1.0e9
    assert bench._traffic(table, "rows_pass2", [{"pass": 2, "chosen": "default"}]) == 1.0e9
    assert bench._traffic(table, "rows_pass2", [{"pass": 2, "chosen": "rows_cluster2"}]) is None
    assert bench._traffic(table, "rows_pass2", [{"pass": 4, "chosen": "rows_cluster2"}]) == 1.0e9
    assert bench._traffic(table, "rows_pass4", None) is None
