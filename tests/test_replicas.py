"""The multi-GPU form is independent replicas (the job does not shard): the
bench times each rank's replica, takes the maximum over ranks and reports the
units of all ranks over that time.  This runs the same reduction on two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_s = 0.5 + rank                  # rank 1 is the slow one
        t, value = bench.replica_value(local_s, 1000.0, dist, "cpu")
        out.put((rank, t, value))
    finally:
        dist.destroy_process_group()


def test_replica_value_is_max_over_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in got:
        assert t == 1.5                       # the slower replica's time
        assert value == pytest.approx(2 * 1000.0 / 1.5)


def test_replica_value_single_process():
    sys.path.insert(0, ROOT)
    import bench
    t, value = bench.replica_value(2.0, 10.0)
    assert (t, value) == (2.0, 5.0)
