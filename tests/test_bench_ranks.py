"""The multi-rank reduction of bench.py on CPU: two gloo ranks (replicas) with
different step times; the job time is the slowest rank's and the throughput
counts both ranks' cells."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    dist.barrier()
    ms, value = bench.job_throughput(10.0 * (rank + 1), 1000, 4, world, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    ms, value = res[0]
    assert ms == 20.0                                   # the slower rank
    assert value == pytest.approx(1000 * 4 * 2 / 0.020 / 1e6)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.job_throughput(5.0, 100, 2, 1, "cpu")
    assert ms == 5.0 and value == pytest.approx(100 * 2 / 0.005 / 1e6)
