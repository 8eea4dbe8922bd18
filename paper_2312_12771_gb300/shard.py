"""Monolithic macro Newton with the RVEs spread over processes (one GPU each).

Section 4.1: the micro block L of the monolithic system is block diagonal
over the macro Gauss points, so the RVEs of different Gauss points never
couple; only the macro system does.  Each process owns a contiguous range of
macro elements and the RVEs of their Gauss points, solves those RVEs,
assembles the macro tangent K and residual R from its own Gauss points only,
and one sum over the processes (an all-reduce of K and of R) gives every
process the same macro system.  Every process then solves it and applies the
same update to the nodal positions, and updates its own RVEs' fluctuations.

All arithmetic runs in libfe2 (macro assembly, band Cholesky, RVE solves);
this module holds the partition, the loop control and the reductions, which
go through a communicator object (``TorchComm`` over torch.distributed: NCCL
between GPUs, gloo on the host).
"""
from __future__ import annotations

import numpy as np

from .driver import NewtonLog


def partition(nelem, world, rank):
    """Macro elements [e0, e1) owned by `rank`: contiguous blocks whose sizes
    differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return rank * nelem // world, (rank + 1) * nelem // world


def gauss_range(nelem, world, rank, d):
    """Macro Gauss points b = 2^d e + q of the elements `rank` owns."""
    e0, e1 = partition(nelem, world, rank)
    return (1 << d) * e0, (1 << d) * e1


class TorchComm:
    """Sums and maxima over the processes of a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce_sum_(self, t):
        """In place: t <- sum over the processes of t."""
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t

    def allreduce_max(self, x):
        import torch
        dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())


class ShardedFE2:
    """The load-stepped monolithic Newton of ``driver.MonolithicFE2`` (Dirac
    basis) with this process's share of the RVEs.  `batch` holds the RVEs of
    the Gauss points ``gauss_range(len(conn), comm.world, comm.rank, d)``, in
    Gauss-point order."""

    def __init__(self, ctx, X, conn, fixed, batch, comm):
        import torch
        if getattr(ctx, "nq", 1) != 1:
            raise ValueError("the sharded Newton takes Dirac-basis RVEs")
        self.t = torch
        self.ctx = ctx
        self.comm = comm
        self.X = np.asarray(X, float)
        self.fixed = np.asarray(fixed, np.uint8)
        d = ctx.dim
        self.d = d
        nelem = len(conn)
        self.ngp = (1 << d) * nelem
        self.g0, self.g1 = gauss_range(nelem, comm.world, comm.rank, d)
        if batch.nrve != self.g1 - self.g0:
            raise ValueError(f"rank {comm.rank} owns {self.g1 - self.g0} Gauss points, got {batch.nrve} RVEs")
        ctx.macro_setup(self.X, conn, self.fixed)
        self.ids = ctx.register_batch(batch)
        dev, f64 = "cuda", torch.float64
        dd = d * d
        self.Fbar = torch.zeros((self.ngp, d, d), dtype=f64, device=dev)
        self.dFbar = torch.zeros_like(self.Fbar)
        # full-size stress / tangent arrays: zero outside this process's Gauss points
        self.sig = torch.zeros((self.ngp, dd), dtype=f64, device=dev)
        self.Cb = torch.zeros((self.ngp, dd, dd), dtype=f64, device=dev)
        self.Pbar = torch.zeros((self.ngp, dd), dtype=f64, device=dev)
        self.outs = ctx._outs(batch.nrve)
        nfree, kd = ctx.macro_system_size()
        self.K = torch.zeros((nfree, kd + 1), dtype=f64, device=dev)
        self.R = torch.zeros(nfree, dtype=f64, device=dev)
        self.rn = torch.zeros(2, dtype=f64, device=dev)
        self.rnm = torch.zeros(batch.nrve, dtype=f64, device=dev)
        self.mstatus = torch.zeros(1, dtype=torch.int32, device=dev)

    def state(self):
        """This process's Gauss points: Fbar, Pbar, sigma_eff, Cbar (host arrays)."""
        sl = slice(self.g0, self.g1)
        sig, Cb, st, err = self.outs
        return dict(Fbar=self.Fbar[sl].cpu().numpy().copy(), Pbar=self.Pbar[sl].cpu().numpy().copy(),
                    sigma_eff=sig.cpu().numpy().copy(), Cbar=Cb.cpu().numpy().copy(),
                    status=st.cpu().numpy().copy())

    def load_step(self, Fk, step, tol_macro=1e-9, tol_micro=1e-9, maxit=25, log=None, F_prev=None):
        ctx, comm = self.ctx, self.comm
        sl = slice(self.g0, self.g1)
        if F_prev is not None:
            q = ctx.macro_get_positions() + self.X @ (np.asarray(Fk) - np.asarray(F_prev)).T
            ctx.macro_set_positions(q)
        ctx.macro_set_positions(self.X @ np.asarray(Fk).T, which=self.fixed)
        sig, Cb, st, err = self.outs
        for it in range(maxit):
            ctx.macro_gradients(self.Fbar)
            ctx.rve_solve(self.ids, self.Fbar[sl], out=self.outs)
            if log is not None:
                log.rve_solve_calls += 1
            self.sig[sl].copy_(sig)
            self.Cb[sl].copy_(Cb)
            ctx.rve_average_stress(self.ids, self.Pbar[sl])
            ctx.macro_assemble(self.Pbar, None, None, self.R)
            comm.allreduce_sum_(self.R)
            ctx.macro_norm(self.R, self.rn[0:1])
            ctx.rve_residual_norm(self.ids, self.rnm)
            self.t.cuda.current_stream().synchronize()
            rmac = float(self.rn[0].item())
            rmic = comm.allreduce_max(float(self.rnm.max().item()) if len(self.ids) else 0.0)
            bad = comm.allreduce_max(float((st != 0).sum().item()))
            if log is not None:
                log.history.append((step, it, rmac, rmic))
            if bad:
                raise RuntimeError(f"RVEs failed on some process (status {np.unique(st.cpu().numpy())} here)")
            if rmac < tol_macro and rmic < tol_micro:
                if log is not None:
                    log.iters.append(it)
                return it
            if rmac > 1e10 or not np.isfinite(rmac):
                if log is not None:
                    log.failed = True
                raise RuntimeError(f"macro residual {rmac:.3e}: Newton diverged")
            ctx.macro_assemble(self.sig, self.Cb, self.K, self.R)
            comm.allreduce_sum_(self.K)
            comm.allreduce_sum_(self.R)
            ctx.macro_solve_assembled(self.K, self.R, self.dFbar, self.rn[1:2], self.mstatus)
            ctx.macro_step(self.ids, self.dFbar[sl])
        raise RuntimeError("macro Newton did not converge")

    def run(self, F_final, n_steps, predictor=False, log=None, traction=None, **kw):
        """As ``MonolithicFE2.run``; the surface load (if any) is held by rank 0
        alone, so that the summed residual counts it once."""
        log = NewtonLog() if log is None else log
        F_final = np.asarray(F_final, float)
        I = np.eye(self.d)
        F_prev = I
        for k in range(1, n_steps + 1):
            Fk = I + (k / n_steps) * (F_final - I)
            if traction is not None and self.comm.rank == 0:
                self.ctx.macro_set_edge_load(traction[0], traction[1], k / n_steps)
            self.load_step(Fk, k, log=log, F_prev=F_prev if predictor else None, **kw)
            F_prev = Fk
        return log
