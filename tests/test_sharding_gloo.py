"""The multi-GPU bench path (one process per GPU, RVEs sharded by rank, no
collective on the data path, max-over-ranks timing) exercised on CPU with the
gloo backend, world size 2."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2312_12771_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank builds its own shard of independent RVEs (different seeds)
    b = W.fiber_batch(8, 4, seed=W.GLOBAL_SEED + rank)
    t = float(10 + 5 * rank)                       # a per-rank elapsed time
    tmax = bench.max_over_ranks(t, True)           # the bench's max-over-ranks timing
    n = torch.tensor([b.nrve], dtype=torch.int64)
    dist.all_reduce(n)                             # total units processed
    out[rank] = (float(tmax), int(n.item()), float(b.mat[:, 0, 1].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_max_timing():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0            # both ranks see the max
    assert res[0][1] == res[1][1] == 16              # whole-job units
    assert res[0][2] != res[1][2]                    # shards differ (independent RVEs)
    # the bench's value: whole-job units over the max time
    assert 16 * 1 / (15.0 * 1e-3) == pytest.approx(1066.67, rel=1e-4)


def test_rank_workloads_are_disjoint_seeds():
    a = bench.workload(4, 4, seed=W.GLOBAL_SEED + 0)
    b = bench.workload(4, 4, seed=W.GLOBAL_SEED + 1)
    assert not np.allclose(a.mat, b.mat)
