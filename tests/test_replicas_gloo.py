"""bench.py's multi-GPU path runs independent replicas (the solve does not shard): the only
cross-rank steps are a barrier and the max/sum reductions of times and work.  Checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import importlib
    import sys

    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    bench = importlib.import_module("bench")
    r, w, _ = bench.dist_setup(None)
    bench.barrier(w)
    t = bench.reduce_max(1.0 + r, w)           # per-rank timed region
    u = bench.reduce_sum(10.0 * (1 + r), w)    # per-rank cell updates
    out[r] = (r, w, t, u, u / t)
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_like_the_driver():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rank, w, t, u, v = res[r]
        assert w == 2 and t == 2.0 and u == 30.0 and v == 15.0
