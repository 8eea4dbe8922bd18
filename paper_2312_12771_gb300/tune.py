"""Measured choice of the launch configuration (the library's own autotuner).

What the kernels leave open is chosen by timing the candidates on the GPU
at hand, on the caller's own RVEs, and the choice is cached in a JSON file
keyed by device name, dimension, precision and the multiset of mesh sizes:

* ``tune_factor``: the band factor kernel of a context (CUDA cores with
  panel phases, CUDA cores with the pipelined panel chain, tensor cores),
  timed as whole RVE solves (CUDA events) and checked to give the same
  statuses;
* ``tune_server``: the serving configuration (batch limit, lane count,
  mixed-size batches), timed as the burst capacity of a request stream;
  optionally the smallest batches within a given fraction of the best
  capacity, for shorter waits.

The panel width (32) and the one RVE per CTA are fixed by the kernels'
design and are not tuned.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

DEFAULT_SERVER = {"max_batch": 512, "lanes": 2, "mixed": False}


def cache_key(kind, d, precision, sizes):
    import torch
    name = torch.cuda.get_device_name(torch.cuda.current_device())
    Ns = ",".join(f"{N}x{c}" for N, c in zip(*np.unique(np.asarray(sizes), return_counts=True)))
    return f"{kind}|{name}|d{d}|{precision}|{Ns}"


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def _store(path, key, value):
    if not path:
        return
    data = _load(path)
    data[key] = value
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_solves(ctx, ids, F, reps):
    import torch
    outs = ctx._outs(len(ids))
    ctx.rve_solve(ids, F, out=outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        ctx.rve_solve(ids, F, out=outs)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, outs[2].cpu().numpy().copy()


def tune_factor(batch, precision="mixed", kernels=("cuda_core", "cuda_core_pipelined", "tensor_core"), reps=3,
                cache=None, **ctx_kw):
    """Time whole RVE solves of `batch` with each band factor kernel; returns
    {"best": kernel, "ms": {kernel: ms per solve of the batch}} (from the
    cache when present)."""
    import torch
    from .fe2 import Fe2Context
    key = cache_key("factor", batch.d, precision, batch.N)
    hit = _load(cache).get(key)
    if hit:
        return dict(hit, cached=True)
    F = torch.tensor(batch.Fbar, device="cuda")
    ms, status = {}, {}
    for kern in kernels:
        ctx = Fe2Context(dim=batch.d, precision=precision, factor=kern, **ctx_kw)
        ids = ctx.register_batch(batch)
        ms[kern], status[kern] = _time_solves(ctx, ids, F, reps)
        ctx.close()
    ref = status[kernels[0]]
    ok = [k for k in kernels if np.array_equal(status[k], ref)]
    best = min(ok, key=lambda k: ms[k])
    res = {"best": best, "ms": {k: round(v, 4) for k, v in ms.items()}}
    _store(cache, key, res)
    return dict(res, cached=False)


def burst_capacity(ctx, ids, Fbar, max_batch, lanes, mixed, reps=2):
    """RVE solves/s of the server draining a burst of one request per RVE."""
    from .serve import Server
    srv = Server(ctx, max_batch=max_batch, lanes=lanes, mixed=mixed)
    srv.submit(ids, Fbar)
    srv.drain()                     # first burst: workspaces, captured graphs
    best = 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        srv.submit(ids, Fbar)
        _, _, _, st, _ = srv.drain()
        dt = time.perf_counter() - t0
        if (st != 0).any():
            srv.close()
            raise RuntimeError("a request failed while tuning")
        best = max(best, len(ids) / dt)
    srv.close()
    return best


def choose_server(table, slack=0.0):
    """The configuration picked from a measured table: among the rows whose
    capacity is within `slack` of the best, the smallest batch limit, then the
    fewest lanes, then the highest capacity.  Returns (row, best capacity)."""
    top = max(r["capacity"] for r in table)
    near = [r for r in table if r["capacity"] >= (1.0 - slack) * top]
    return min(near, key=lambda r: (r["max_batch"], r["lanes"], -r["capacity"])), top


def tune_server(ctx, ids, Fbar, sizes, max_batches=(128, 256, 512, 1024), lanes=(2, 3, 4),
                mixed=(False, True), cache=None, slack=0.0):
    """Burst capacity of every (max_batch, lanes, mixed) candidate on the
    caller's RVEs; returns {"best": config, "capacity": its solves/s,
    "max_capacity": the best solves/s, "default": solves/s of DEFAULT_SERVER,
    "table": [...]}.  Candidates within `slack` (a fraction) of the best
    capacity are ranked by batch limit, then lane count: smaller batches and
    fewer concurrent ones keep a request's wait shorter."""
    key = cache_key("server", ctx.dim, ctx.precision, sizes) + f"|slack{slack:g}"
    hit = _load(cache).get(key)
    if hit:
        return dict(hit, cached=True)
    table = []
    for mb in max_batches:
        for ln in lanes:
            for mx in mixed:
                cap = burst_capacity(ctx, ids, Fbar, mb, ln, mx)
                table.append({"max_batch": mb, "lanes": ln, "mixed": mx, "capacity": round(cap, 1)})
    best, top = choose_server(table, slack)
    dflt = next((r["capacity"] for r in table if r["max_batch"] == DEFAULT_SERVER["max_batch"] and
                 r["lanes"] == DEFAULT_SERVER["lanes"] and r["mixed"] == DEFAULT_SERVER["mixed"]), None)
    if dflt is None:
        dflt = round(burst_capacity(ctx, ids, Fbar, **DEFAULT_SERVER), 1)
    res = {"best": {k: best[k] for k in ("max_batch", "lanes", "mixed")}, "capacity": best["capacity"],
           "max_capacity": top, "slack": slack, "default": dflt, "table": table}
    _store(cache, key, res)
    return dict(res, cached=False)
