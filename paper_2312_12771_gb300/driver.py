"""FE^2 Newton drivers over the C ABI: the monolithic scheme (Section 4.2,
Eq. (solution2)) and the classical staggered scheme (Section 4.1).

The loop control lives here; every arithmetic step is a libfe2 kernel:
macro gradients, the fused RVE solve (S1-S6), the volume-averaged stress and
micro residual norms, the macro assembly + band solve (S7) and the
fluctuation update w~ <- w~ - (x_r + X_M : dFbar).  The staggered scheme
instead brings every RVE to micro equilibrium (inner Newton: the same update
with dFbar = 0) before each macro iteration.  Load stepping follows
Section 5.2: the Dirichlet data are applied in n_l increments and each load
step starts from the previous converged state.  A step fails when the macro
residual exceeds 1e10 (the failure criterion of Section 5.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def macro_mesh(nx, ny, Lx=1.0, Ly=1.0):
    """Structured Q4 mesh of [0,Lx]x[0,Ly]; boundary nodes flagged as Dirichlet."""
    xs = np.linspace(0.0, Lx, nx + 1)
    ys = np.linspace(0.0, Ly, ny + 1)
    X = np.array([[x, y] for y in ys for x in xs])
    conn = []
    for ey in range(ny):
        for ex in range(nx):
            n0 = ex + (nx + 1) * ey
            conn.append([n0, n0 + 1, n0 + nx + 1, n0 + nx + 2])
    conn = np.array(conn, dtype=np.int32)
    on_bnd = (np.abs(X[:, 0]) < 1e-12) | (np.abs(X[:, 1]) < 1e-12) | \
        (np.abs(X[:, 0] - Lx) < 1e-12) | (np.abs(X[:, 1] - Ly) < 1e-12)
    fixed = np.repeat(on_bnd, 2).astype(np.uint8)
    return X, conn, fixed


def macro_mesh3(nx, ny, nz, Lx=1.0, Ly=1.0, Lz=1.0):
    """Structured Hex8 mesh of [0,Lx]x[0,Ly]x[0,Lz] (nodes x fastest, local node
    a = a_x + 2 a_y + 4 a_z); boundary nodes flagged as Dirichlet."""
    g = np.meshgrid(np.linspace(0.0, Lx, nx + 1), np.linspace(0.0, Ly, ny + 1), np.linspace(0.0, Lz, nz + 1),
                    indexing="ij")
    X = np.stack([g[0].ravel(order="F"), g[1].ravel(order="F"), g[2].ravel(order="F")], axis=1)
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ex, ey, ez = ex.ravel(order="F"), ey.ravel(order="F"), ez.ravel(order="F")
    conn = np.stack([(ex + (a & 1)) + (nx + 1) * ((ey + ((a >> 1) & 1)) + (ny + 1) * (ez + ((a >> 2) & 1)))
                     for a in range(8)], axis=1).astype(np.int32)
    L = np.array([Lx, Ly, Lz])
    on_bnd = ((np.abs(X) < 1e-12) | (np.abs(X - L) < 1e-12)).any(axis=1)
    fixed = np.repeat(on_bnd, 3).astype(np.uint8)
    return X, conn, fixed


@dataclass
class NewtonLog:
    iters: list = field(default_factory=list)      # Newton iterations per load step
    history: list = field(default_factory=list)    # (step, it, ||R_macro||, max ||r_m||)
    failed: bool = False
    micro_iters: int = 0                           # staggered: inner micro Newton updates (all RVEs at once)
    rve_solve_calls: int = 0                       # batched fe2_rve_solve calls
    micro_history: list = field(default_factory=list)  # staggered: (step, it, max ||r_m||) before each update


class MonolithicFE2:
    """Macro Q4 (2D) or Hex8 (3D) problem with one RVE per macro Gauss point
    (b = 2^d e + q), or, on a 2D context with the piecewise-constant basis, one
    element RVE per macro element (Eqs. (constSolution1), (constSolution2))
    whose four Gauss points are weighted by eta_q / sum eta."""

    def __init__(self, ctx, X, conn, fixed, batch):
        import torch
        self.t = torch
        self.ctx = ctx
        self.X = np.asarray(X, float)
        self.fixed = np.asarray(fixed, np.uint8)
        d = ctx.dim
        self.d = d
        ngp = (1 << d) * len(conn)
        nrve = ngp // getattr(ctx, "nq", 1)
        if batch.nrve != nrve:
            raise ValueError(f"need {nrve} RVEs ({'macro elements' if nrve != ngp else 'macro Gauss points'}), "
                             f"got {batch.nrve}")
        ctx.macro_setup(self.X, conn, self.fixed)
        self.ids = ctx.register_batch(batch)
        self.maxnm = int(max(d * (int(N) ** d - 1) for N in batch.N))
        dev = "cuda"
        f64 = torch.float64
        self.Fbar = torch.zeros((ngp, d, d), dtype=f64, device=dev)
        self.dFbar = torch.zeros_like(self.Fbar)
        self.Pbar = torch.zeros((ngp, d * d), dtype=f64, device=dev)
        self.outs = ctx._outs(nrve)
        self.rn = torch.zeros(2, dtype=f64, device=dev)
        self.rnm = torch.zeros(nrve, dtype=f64, device=dev)
        if nrve != ngp:
            eta = torch.zeros(ngp, dtype=f64, device=dev)
            ctx.macro_gradients(self.Fbar, eta)
            e = eta.cpu().numpy().reshape(nrve, 4)
            ctx.rve_set_quad_weights(self.ids, e / e.sum(axis=1, keepdims=True))
        self.mstatus = torch.zeros(1, dtype=torch.int32, device=dev)
        self.zero_dF = torch.zeros_like(self.Fbar)
        self.ngp = ngp

    def state(self):
        """Current per-Gauss-point Fbar, Pbar, sigma_eff, Cbar (host arrays)."""
        sig, Cb, st, err = self.outs
        return dict(Fbar=self.Fbar.cpu().numpy().copy(), Pbar=self.Pbar.cpu().numpy().copy(),
                    sigma_eff=sig.cpu().numpy().copy(), Cbar=Cb.cpu().numpy().copy(),
                    status=st.cpu().numpy().copy(), err=err.cpu().numpy().copy())

    def set_traction(self, nodes, T, scale):
        """Surface load of the current load step (Neumann term of Eq. (weakMech)):
        the traction T on the boundary polyline `nodes`, times `scale`; the
        library forms the nodal forces."""
        self.ctx.macro_set_edge_load(nodes, T, scale)

    def load_step(self, Fk, step, tol_macro=1e-9, tol_micro=1e-9, maxit=25, log=None, F_prev=None):
        """One load step.  The previous converged state is the start value
        (Section 5.2); with ``F_prev`` given, the affine increment
        (Fk - F_prev) X is added to every node first (affine predictor), so
        that the Dirichlet increment does not distort only the boundary
        elements of a fine macro mesh."""
        ctx = self.ctx
        if F_prev is not None:
            q = ctx.macro_get_positions() + self.X @ (np.asarray(Fk) - np.asarray(F_prev)).T
            ctx.macro_set_positions(q)
        q_fixed = self.X @ np.asarray(Fk).T
        ctx.macro_set_positions(q_fixed, which=self.fixed)
        sig, Cb, st, err = self.outs
        for it in range(maxit):
            ctx.macro_gradients(self.Fbar)
            ctx.rve_solve(self.ids, self.Fbar, out=self.outs)
            if log is not None:
                log.rve_solve_calls += 1
            ctx.rve_average_stress(self.ids, self.Pbar)
            ctx.macro_residual(self.Pbar, self.rn[0:1])
            ctx.rve_residual_norm(self.ids, self.rnm)
            self.t.cuda.current_stream().synchronize()
            rmac = float(self.rn[0].item())
            rmic = float(self.rnm.max().item())
            bad = int((st != 0).sum().item())
            if log is not None:
                log.history.append((step, it, rmac, rmic))
            if bad:
                raise RuntimeError(f"{bad} RVEs failed (status {np.unique(st.cpu().numpy())})")
            if rmac < tol_macro and rmic < tol_micro:
                if log is not None:
                    log.iters.append(it)
                return it
            if rmac > 1e10 or not np.isfinite(rmac):
                if log is not None:
                    log.failed = True
                raise RuntimeError(f"macro residual {rmac:.3e}: Newton diverged")
            ctx.macro_solve(sig, Cb, self.dFbar, self.rn[1:2], self.mstatus)
            ctx.macro_step(self.ids, self.dFbar)
        raise RuntimeError("macro Newton did not converge")

    def load_step_staggered(self, Fk, step, tol_macro=1e-9, tol_micro=1e-11, maxit=25, maxit_micro=30, log=None,
                            F_prev=None, micro_start="predicted"):
        """One load step of the classical staggered scheme (Section 4.1): in
        every macro iteration all RVEs are first brought to micro equilibrium
        at their current Fbar (inner Newton w~ <- w~ - x_r, i.e. the micro
        update with dFbar = 0, until max ||r_m|| < tol_micro); Pbar and the
        condensed tangent at that equilibrium then give the macro residual and
        stiffness (Eq. (solution1)); after the macro step the micro states follow
        Eq. (reduction), dw~ = -X_M : dFbar, before they are re-equilibrated.
        With ``micro_start`` = "last_converged" every inner Newton instead starts
        from the micro states of the last converged load step (a device-side
        snapshot, fe2_rve_w_copy): the reading of Section 5.2, Table 2.""" 
        ctx = self.ctx
        if F_prev is not None:
            q = ctx.macro_get_positions() + self.X @ (np.asarray(Fk) - np.asarray(F_prev)).T
            ctx.macro_set_positions(q)
        ctx.macro_set_positions(self.X @ np.asarray(Fk).T, which=self.fixed)
        sig, Cb, st, err = self.outs
        restart = micro_start == "last_converged"
        for it in range(maxit):
            ctx.macro_gradients(self.Fbar)
            if restart:
                ctx.w_copy(self.ids, self.wsnap, to_buf=False)
            for mit in range(maxit_micro):
                ctx.rve_solve(self.ids, self.Fbar, out=self.outs)
                ctx.rve_residual_norm(self.ids, self.rnm)
                self.t.cuda.current_stream().synchronize()
                if log is not None:
                    log.rve_solve_calls += 1
                    log.micro_history.append((step, it, float(self.rnm.max().item())))
                bad = int((st != 0).sum().item())
                if bad:
                    if log is not None:
                        log.failed = True
                    raise RuntimeError(f"{bad} RVEs failed (status {np.unique(st.cpu().numpy())})")
                rmic = float(self.rnm.max().item())
                if rmic < tol_micro:
                    break
                if not np.isfinite(rmic) or rmic > 1e10:
                    if log is not None:
                        log.failed = True
                    raise RuntimeError(f"micro residual {rmic:.3e}: inner Newton diverged")
                ctx.macro_step(self.ids, self.zero_dF)
                if log is not None:
                    log.micro_iters += 1
            else:
                if log is not None:
                    log.failed = True
                raise RuntimeError("micro Newton did not converge")
            ctx.rve_average_stress(self.ids, self.Pbar)
            ctx.macro_residual(self.Pbar, self.rn[0:1])
            self.t.cuda.current_stream().synchronize()
            rmac = float(self.rn[0].item())
            if log is not None:
                log.history.append((step, it, rmac, rmic))
            if rmac < tol_macro:
                if log is not None:
                    log.iters.append(it)
                if restart:
                    ctx.w_copy(self.ids, self.wsnap, to_buf=True)
                return it
            if rmac > 1e10 or not np.isfinite(rmac):
                if log is not None:
                    log.failed = True
                raise RuntimeError(f"macro residual {rmac:.3e}: Newton diverged")
            ctx.macro_solve(sig, Cb, self.dFbar, self.rn[1:2], self.mstatus)
            if not restart:
                # Eq. (reduction): dw~ = -X_M : dFbar (x_r vanishes at micro equilibrium)
                ctx.macro_step(self.ids, self.dFbar)
        if log is not None:
            log.failed = True
        raise RuntimeError("macro Newton did not converge")

    def run(self, F_final, n_steps, predictor=False, scheme="monolithic", log=None, traction=None, **kw):
        """Load-stepped solve; ``scheme`` is "monolithic" (Section 4.2) or
        "staggered" (Section 4.1).  Step k applies the Dirichlet data of
        F_k = I + k/n (F_final - I) and, with ``traction`` = (boundary nodes,
        T), the surface load k/n T on that edge (Section 5.2: T_k = k T / n_l).
        A failing step raises; ``log`` (if given) keeps what was recorded up
        to the failure."""
        log = NewtonLog() if log is None else log
        step_fn = self.load_step if scheme == "monolithic" else self.load_step_staggered
        if kw.get("micro_start") == "last_converged":   # snapshot of the start state
            self.wsnap = self.t.zeros((len(self.ids), self.maxnm), dtype=self.t.float64, device="cuda")
            self.ctx.w_copy(self.ids, self.wsnap, to_buf=True)
        F_final = np.asarray(F_final, float)
        I = np.eye(self.d)
        F_prev = I
        for k in range(1, n_steps + 1):
            Fk = I + (k / n_steps) * (F_final - I)
            if traction is not None:
                self.set_traction(traction[0], traction[1], k / n_steps)
            step_fn(Fk, k, log=log, F_prev=F_prev if predictor else None, **kw)
            F_prev = Fk
        return log
