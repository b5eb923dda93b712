"""Replica timing reductions across two CPU processes (torch.distributed, gloo, world size 2).

Each rank plays one GPU of a multi-GPU run: it reports its own work and time; the whole-job
throughput must be the total work over the slowest rank's time, identical on every rank.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2308_08447_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    replicas.barrier()
    units = 1000.0 * (rank + 1)          # rank 0: 1000 cells, rank 1: 2000 cells
    seconds = 2.0 + rank                 # rank 1 is the slowest
    thr, t, total = replicas.job_throughput(units, seconds)
    with open(os.path.join(out_dir, "r%d.txt" % rank), "w") as fh:
        fh.write("%r %r %r %r" % (thr, t, total, replicas.max_over_ranks(rank)))
    dist.destroy_process_group()


def test_job_throughput_two_ranks(tmp_path):
    import sys

    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    vals = [open(tmp_path / ("r%d.txt" % r)).read().split() for r in range(2)]
    assert vals[0] == vals[1]
    thr, t, total, mx = (float(v) for v in vals[0])
    assert total == 3000.0 and t == 3.0 and thr == 1000.0 and mx == 1.0


def test_single_process_is_identity():
    from paper_2308_08447_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(10.0, 2.0) == (5.0, 2.0, 10.0)
