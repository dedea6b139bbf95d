"""The multi-process side of bench.py on the CPU (gloo, two ranks): the
replicas' whole-job time is the slowest rank's, and the job's throughput is
world x per-rank iterations over it.  No GPU: the GPU path runs the same
functions with NCCL."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    job = bench.whole_job_ms(ms, w, torch.device("cpu"))
    out[rank] = (r, w, local, job, bench.job_value(w, 52, job))
    dist.destroy_process_group()


def test_whole_job_time_is_the_slowest_rank():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        r, w, local, job, value = res[rank]
        assert (r, w, local) == (rank, world, rank)
        assert job == 15.0
        assert value == pytest.approx(2 * 52 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_ms(12.5, 1, None) == 12.5
    assert bench.job_value(1, 52, 26.0) == pytest.approx(2000.0)
