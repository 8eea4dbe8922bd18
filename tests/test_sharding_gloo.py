"""Multi-process paths on the host with the gloo backend, world size 2.

1. The bench's sharded timing: each rank its own RVEs, max-over-ranks time
   (``bench.max_over_ranks``), whole-job units.
2. The sharded macro Newton's partition and reduction (``shard.partition``,
   ``shard.gauss_range``, ``shard.TorchComm``): each rank forms the macro
   system of Section 3, Eq. (linSys2) from its own Gauss points with the
   oracle (the stresses and tangents of the other ranks' points are zero), the
   product's communicator sums them, and the sum equals the oracle's system
   over all Gauss points; the partition covers every element once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import fe2_oracle as O
from paper_2312_12771_gb300 import shard
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


def _macro_case(d):
    """A small macro mesh with seeded per-Gauss-point stresses and major-symmetric tangents."""
    if d == 2:
        X, conn, _ = O.macro_mesh(3, 2)
    else:
        X, conn, _ = O.macro_mesh3(2, 2, 1)
    grads, etas, _ = O.macro_gauss(X, conn)
    rng = np.random.default_rng(40 + d)
    ngp = len(etas)
    stress = rng.standard_normal((ngp, d, d))
    A = rng.standard_normal((ngp, d * d, d * d))
    Cbar = A + A.transpose(0, 2, 1)
    return conn, grads, etas, stress, Cbar


def _shard_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = shard.TorchComm()
    res = {}
    for d in (2, 3):
        conn, grads, etas, stress, Cbar = _macro_case(d)
        g0, g1 = shard.gauss_range(len(conn), comm.world, comm.rank, d)
        s_loc, C_loc = np.zeros_like(stress), np.zeros_like(Cbar)
        s_loc[g0:g1], C_loc[g0:g1] = stress[g0:g1], Cbar[g0:g1]
        K, R = O.macro_system(conn, grads, etas, s_loc, C_loc, d)
        Kt, Rt = torch.tensor(K), torch.tensor(R)
        comm.allreduce_sum_(Kt)
        comm.allreduce_sum_(Rt)
        res[d] = (Kt.numpy().copy(), Rt.numpy().copy(), (g0, g1), comm.allreduce_max(float(rank)))
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_macro_system_reduces_to_the_full_system():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for d in (2, 3):
        conn, grads, etas, stress, Cbar = _macro_case(d)
        K, R = O.macro_system(conn, grads, etas, stress, Cbar, d)
        for rank in (0, 1):
            Kr, Rr, _, mx = res[rank][d]
            assert np.abs(Kr - K).max() <= 1e-12 * np.abs(K).max()
            assert np.abs(Rr - R).max() <= 1e-12 * np.abs(R).max()
            assert mx == 1.0
        # the two ranks' Gauss points tile [0, ngp) without overlap
        (a0, a1), (b0, b1) = res[0][d][2], res[1][d][2]
        assert a0 == 0 and a1 == b0 and b1 == len(etas) and a1 > a0 and b1 > b0


@pytest.mark.parametrize("nelem,world", [(1, 1), (7, 2), (8, 3), (1024, 8), (5, 5)])
def test_partition_covers_every_element_once(nelem, world):
    got = [shard.partition(nelem, world, r) for r in range(world)]
    assert got[0][0] == 0 and got[-1][1] == nelem
    assert all(got[r][1] == got[r + 1][0] for r in range(world - 1))
    sizes = [b - a for a, b in got]
    assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.partition(nelem, world, world)


def test_rank_workloads_are_disjoint_seeds():
    a = bench.workload(4, 4, seed=W.GLOBAL_SEED + 0)
    b = bench.workload(4, 4, seed=W.GLOBAL_SEED + 1)
    assert not np.allclose(a.mat, b.mat)
