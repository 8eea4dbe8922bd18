"""The sharded macro Newton on one GPU (Section 4.1: only the macro system
couples the RVEs of different Gauss points).

1. fe2_macro_assemble + fe2_macro_solve_assembled on one process equal
   fe2_macro_solve bit for bit.
2. Two ranks emulated by two host threads, each with its own context and half
   of the macro elements' RVEs, their K and R summed by an in-process
   all-reduce: the same Newton iterations, nodal positions and converged
   Pbar / Cbar as the single-context monolithic Newton, and as the oracle's.
   (The ranks wait for each other on the host only; no kernel waits on
   another.)"""
import threading

import numpy as np
import pytest

from oracle import fe2_oracle as O
from paper_2312_12771_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12771_gb300 import build
    build.build()
    return t


def test_split_macro_update_equals_fused(torch):
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    from paper_2312_12771_gb300.fe2 import Fe2Context
    X, conn, fixed = macro_mesh(3, 2)
    b = W.inclusion_batch(24, 6, stretch=1.0)
    out = []
    for split in (False, True):
        ctx = Fe2Context(dim=2, precision="fp64")
        fe = MonolithicFE2(ctx, X, conn, fixed, b)
        # a smooth non-affine deformation of every node: finite, positive Jacobians
        q = X @ np.diag([1.05, 0.98]).T + 0.01 * np.sin(3.0 * X[:, ::-1])
        ctx.macro_set_positions(q)
        ctx.macro_gradients(fe.Fbar)
        sig, Cb, st, err = ctx.rve_solve(fe.ids, fe.Fbar)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        dF = torch.zeros_like(fe.Fbar)
        rn = torch.zeros(1, dtype=torch.float64, device="cuda")
        if split:
            nf, kd = ctx.macro_system_size()
            K = torch.zeros((nf, kd + 1), dtype=torch.float64, device="cuda")
            R = torch.zeros(nf, dtype=torch.float64, device="cuda")
            ctx.macro_assemble(sig, Cb, K, R)
            ctx.macro_solve_assembled(K, R, dF, rn)
        else:
            ctx.macro_solve(sig, Cb, dF, rn)
        torch.cuda.synchronize()
        out.append((dF.cpu().numpy(), rn.cpu().numpy(), ctx.macro_get_positions()))
        ctx.close()
    for a, c in zip(out[0], out[1]):
        assert np.isfinite(a).all() and np.array_equal(a, c)


class ThreadComm:
    """In-process all-reduce between host threads (one per emulated rank): the
    sum is formed in rank order by every rank, so all ranks hold the same bits."""

    def __init__(self, shared, rank, world):
        self.sh, self.rank, self.world = shared, rank, world

    def _exchange(self, x):
        import torch
        torch.cuda.synchronize()
        self.sh["slots"][self.rank] = x
        self.sh["barrier"].wait()
        vals = list(self.sh["slots"])
        self.sh["barrier"].wait()
        return vals

    def allreduce_sum_(self, t):
        import torch
        vals = self._exchange(t)
        total = vals[0].clone()
        for v in vals[1:]:
            total += v
        torch.cuda.synchronize()
        self.sh["barrier"].wait()          # every rank has read every slot
        t.copy_(total)
        torch.cuda.synchronize()
        return t

    def allreduce_max(self, x):
        return max(self._exchange(float(x)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_rank_sharded_newton_matches_monolithic_and_oracle(torch, precision):
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    from paper_2312_12771_gb300.fe2 import Fe2Context
    from paper_2312_12771_gb300.shard import ShardedFE2, gauss_range
    N, world = 6, 2
    X, conn, fixed = macro_mesh(3, 2)
    ngp = 4 * len(conn)
    b = W.inclusion_batch(ngp, N, stretch=1.0)
    Ff = np.diag([1.1, 1.0])
    kw = dict(tol_macro=1e-10, tol_micro=1e-10)
    ctx = Fe2Context(dim=2, precision=precision, refine_tol=1e-14, max_refine=2)
    mono = MonolithicFE2(ctx, X, conn, fixed, b)
    log_m = mono.run(Ff, 2, **kw)
    st_m = mono.state()
    q_m = ctx.macro_get_positions()
    ctx.close()

    shared = {"barrier": threading.Barrier(world), "slots": [None] * world}
    results, errors = [None] * world, []

    def rank_main(rank):
        try:
            torch.cuda.set_device(0)
            c = Fe2Context(dim=2, precision=precision, refine_tol=1e-14, max_refine=2)
            g0, g1 = gauss_range(len(conn), world, rank, 2)
            fe = ShardedFE2(c, X, conn, fixed, b.subset(range(g0, g1)), ThreadComm(shared, rank, world))
            log = fe.run(Ff, 2, **kw)
            results[rank] = (log.iters, fe.state(), c.macro_get_positions(), (g0, g1))
            c.close()
        except BaseException as exc:      # reported by the main thread
            errors.append(exc)
            shared["barrier"].abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    assert not errors, errors
    tol = 1e-10 if precision == "fp64" else 1e-8
    for rank in range(world):
        iters, st, q, (g0, g1) = results[rank]
        assert iters == log_m.iters
        assert np.abs(q - q_m).max() <= 1e-11
        for k in range(g1 - g0):
            assert O.rel_err(st["Pbar"][k], st_m["Pbar"][g0 + k]) <= tol
            assert O.rel_err(st["Cbar"][k], st_m["Cbar"][g0 + k]) <= tol
    assert np.array_equal(results[0][2], results[1][2])     # both ranks hold the same positions
    # and the oracle's monolithic scheme
    rves = [dict(N=N, phase=b.phase[k], mat=b.mat[k]) for k in range(ngp)]
    out, iters, q = O.monolithic_fe2(O.macro_mesh(3, 2), rves, Ff, n_steps=2, **kw)
    assert log_m.iters == iters
    assert np.abs(results[0][2] - q).max() <= 1e-11
