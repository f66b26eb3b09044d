"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own seeded 1D batch,
combine their work (sum) and their timed region (the slowest rank) the way a torchrun job
over several GPUs does, with no collective on the data path."""
import os
import socket
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench

    w, desc = bench.make_workload(SimpleNamespace(workload="batch1d", n_batch=8), rank)
    units = bench.rank_reduce(desc["interior_cells"], "sum", world, "cpu")
    ms = bench.rank_reduce(10.0 + rank, "max", world, "cpu")
    out[rank] = (desc["interior_cells"], units, ms, bench.whole_job_mlups(units, 4, ms), list(w.lengths))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_combine_work_and_slowest_time():
    import torch.multiprocessing as mp

    with mp.Manager() as manager:
        out = manager.dict()
        mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[4] != r1[4]  # each rank draws its own batch
    assert r0[1] == r1[1] == r0[0] + r1[0]  # the work of both ranks
    assert r0[2] == r1[2] == 11.0  # the slower rank's time
    assert r0[3] == r1[3] == pytest.approx((r0[0] + r1[0]) * 4 / 0.011 / 1e6)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_reduce(3.5, "max", 1, "cpu") == 3.5
    assert bench.whole_job_mlups(1e6, 10, 1000.0) == pytest.approx(10.0)
