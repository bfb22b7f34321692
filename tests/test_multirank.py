"""The bench's multi-rank bookkeeping on CPU ranks (gloo, world size 2): each
rank computes its own cloud (seed = rank: the clouds differ), the job's time is
the slowest rank's and its work the sum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    from paper_2003_07989_gb300 import inputs as I
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    X = I.noisy_torus(64, seed=r)  # each rank its own cloud
    times = [10.0 + 5.0 * r, 20.0 - r]
    work = [100.0 * (r + 1), 7.0, float(len(X))]
    slow, summed = bench.over_ranks(dist, times, work, "cpu")
    out.put((r, slow, summed, float(X[0, 0])))
    dist.destroy_process_group()


def test_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for r, slow, summed, _ in got:
        assert slow == [15.0, 20.0]                # the slowest rank, per figure
        assert summed == [300.0, 14.0, 128.0]      # work of both ranks
    assert got[0][3] != got[1][3]                  # different clouds per rank
