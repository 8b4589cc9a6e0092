"""The multi-rank path of bench.py (one independent replica per rank, no
data-path collective) on CPU: two gloo ranks each time their own replica;
every rank ends with the slowest rank's time and the whole-job rate counts
the site updates of both replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_s = [1.5, 2.5][rank]
    t = bench.max_over_ranks(local_s, ws, "cpu")
    out[rank] = (t, bench.aggregate_rate(ws, 1000, 64, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, pytest.approx(2 * 1000 * 64 / 2.5))


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.aggregate_rate(1, 10, 5, 2.0) == 25.0
