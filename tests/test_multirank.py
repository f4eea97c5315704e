"""The benchmark's multi-rank logic on CPU (gloo, world size 2): each rank gets its own
field (weak scaling, nothing exchanged on the data path) and times are reduced to the
slowest rank's on every rank."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

import bench
from paper_1801_10277_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    r, n, dist = bench.dist_init("gloo")
    assert (r, n) == (rank, ws) and dist is not None
    # a rank-dependent "time": every rank must see the maximum
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    prob = synth.config(1, seed=bench.rank_field_seed(r))
    out.put((r, t, float(prob.theta[:, 0].sum()), prob.source_pixels()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    assert all(t == 2.5 for _, t, _, _ in res)           # max over ranks, on both ranks
    assert res[0][2] != res[1][2]                       # each rank has its own field
    assert res[0][3] > 0 and res[1][3] > 0


def test_single_rank_needs_no_process_group():
    assert bench.dist_init() == (0, 1, None)
    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    assert bench.rank_field_seed(0) != bench.rank_field_seed(1)
