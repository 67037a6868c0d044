"""The multi-GPU path of bench.py is independent replicas: one pencil per rank
(its f seeded by the rank), no collective on the data path, and the job-wide
numbers formed at the end: max over ranks of the timed region, sum over ranks
of the units processed.  This checks that host logic with world_size 2 on the
gloo backend (CPU only, rendezvous on 127.0.0.1)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    w_, r_, _ = bench.dist_init()
    try:
        t = bench.barrier_max(10.0 + rank, w_)       # timed region: the slowest rank
        n = bench.allreduce_sum(564 + rank, w_)      # units: every rank's
        bench.barrier(w_)
        f = bench.workload(r_).f[:4]
        q.put((r_, w_, t, n, f))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_world_size_2():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, t0, n0, f0), (r1, w1, t1, n1, f1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert t0 == t1 == 11.0            # max over ranks
    assert n0 == n1 == 564 + 565       # sum over ranks
    assert not np.allclose(f0, f1)     # each replica solves its own seeded f
