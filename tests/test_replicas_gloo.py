"""The N > 1 bench path on the host: two ranks over gloo (world_size 2).

Each rank runs an independent replica on its own queries (no collective on
the data path); the timing is the maximum over ranks after a barrier, and the
whole-job value counts every rank's queries."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    import fixtures as fx
    r, w, local, dist = bench.dist_setup(world)
    assert (r, w) == (rank, world) and dist is not None
    bench.barrier(dist)
    # per-rank timings differ; every rank sees the maximum
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    # replicas draw different query sets from the same generator
    X = fx.random_walk(50, 16)
    Q = fx.test_queries(X, 4, seed=fx.SEED_TEST + 1000 * rank)
    out[rank] = (ms, float(Q.sum()))
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]
