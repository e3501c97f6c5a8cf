"""Multi-rank timing aggregation of bench.py on CPU (gloo, world size 2):
the timed region is the maximum over ranks and the rate counts every rank's
units; the reference arm does its work on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, value = bench.whole_job(10.0 * (rank + 1), 1000, 4, dist, "cpu")
    out.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, ms, value in res:
        assert ms == 20.0                           # slowest rank's time
        assert value == pytest.approx(1000 * 4 * 2 / 0.020)


def test_whole_job_single():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job(8.0, 500, 2)
    assert ms == 8.0 and value == pytest.approx(500 * 2 / 0.008)


def test_reference_arm_other_ranks_idle():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.run_reference(None, 1, 2) == 0     # returns before touching args


def test_profile_case_argument(monkeypatch):
    """--profile-case picks one of the benchmark sizes (default d=3 n=17) and
    rejects any other."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--profile-case"])
    assert bench.parse().profile_case == (3, 17)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--profile-case", "5,12"])
    assert bench.parse().profile_case == (5, 12)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    assert bench.parse().profile_case is None
    monkeypatch.setattr(sys, "argv", ["bench.py", "--profile-case", "3,5"])
    with pytest.raises(SystemExit):
        bench.parse()
