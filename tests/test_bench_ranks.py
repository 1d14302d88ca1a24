"""Host logic of bench.py's multi-GPU mode ("replicas only": every rank
solves its own copy of the workload, no collective on the data path), run
as two gloo ranks on the CPU: the whole-job time is the slowest rank's and
the units are summed over ranks; the reference arm prints from rank 0 only."""
import contextlib
import io
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


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, u = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1))
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%r %r" % (t, u))


def test_replica_reduction_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        t, u = open(tmp_path / ("rank%d.txt" % r)).read().split()
        assert float(t) == 11.0 and float(u) == 300.0


def test_reduction_is_identity_on_one_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(5.0, 42) == (5.0, 42)


def test_reference_arm_prints_only_on_rank_zero():
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup = 1, 0
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args(), 2, 1)
    assert buf.getvalue() == ""
