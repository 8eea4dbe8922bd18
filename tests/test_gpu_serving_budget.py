"""Serving under an HBM budget smaller than the RVE states it serves.

The RVEs are defined without device state (fe2_rve_define); the server
admits them batch by batch as memory allows, evicting idle RVEs (their w~
kept on the host) when the budget is full.  With room for a third of the
RVEs at a time, every served result (two rounds of the same stream, the
second after evictions) is bit-identical to the unbudgeted server's and to
each RVE solved alone, and the device bytes held stay within the budget."""
import numpy as np
import pytest

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


def _case():
    n = 24
    sizes = np.array([16, 24] * (n // 2), np.int32)
    b = W.inclusion_batch(n, sizes, stretch=1.04, seed=W.GLOBAL_SEED + 24)
    b.Fbar = W.perturbed_F(b, 25, 0.01)
    rng = np.random.default_rng(26)
    ws = [0.005 / N * rng.standard_normal(2 * (N * N - 1)) for N in sizes]
    return b, ws


def _serve(ctx, ids, F, rounds):
    from paper_2312_12771_gb300.serve import Server
    srv = Server(ctx, max_batch=4, lanes=2)
    outs = []
    for _ in range(rounds):
        tk = srv.submit(ids, F)
        t, sig, Cb, st, _ = srv.drain()
        pos = {int(x): j for j, x in enumerate(tk)}
        order = np.argsort([pos[int(x)] for x in t])
        outs.append((sig[order], Cb[order], st[order]))
    stats = srv.memory_stats()
    srv.close()
    return outs, stats


def test_serving_admits_by_budget_and_matches_unbudgeted_and_alone(torch):
    from paper_2312_12771_gb300.fe2 import Fe2Context
    b, ws = _case()
    n = b.nrve

    def defined(budget, sub=None):
        ctx = Fe2Context(dim=2, precision="mixed", hbm_budget_bytes=budget)
        bb = b if sub is None else b.subset(sub)
        ids = ctx.define_batch(bb)
        for k, i in enumerate(ids):
            ctx.set_w(i, ws[k if sub is None else sub[k]])
        assert all(ctx.resident(i) == 0 for i in ids)
        return ctx, ids

    ctx_a, ids_a = defined(0)
    outs_a, stats_a = _serve(ctx_a, ids_a, b.Fbar, 1)
    ctx_a.close()
    ctx_b, ids_b = defined(0, list(range(4)))
    _, stats_b = _serve(ctx_b, ids_b, b.Fbar[:4], 1)
    ctx_b.close()
    # 24 RVEs took two slabs of 16 slots, 4 RVEs one: the difference is 16 slots
    slot = (stats_a[3] - stats_b[3]) // 16
    lanes = stats_b[3] - 16 * slot
    assert slot > 0 and lanes > 0
    budget = lanes + 8 * slot + slot // 2
    ctx_c, ids_c = defined(budget)
    outs_c, stats_c = _serve(ctx_c, ids_c, b.Fbar, 2)
    admitted, evicted, deferred, held = stats_c
    assert evicted > 0 and admitted > n and held <= budget, stats_c
    for sig, Cb, st in outs_c:
        assert (st == 0).all()
        assert np.array_equal(sig, outs_a[0][0]) and np.array_equal(Cb, outs_a[0][1])
    ctx_c.close()
    # each RVE alone, registered the usual way
    ctx_r = Fe2Context(dim=2, precision="mixed")
    ids_r = ctx_r.register_batch(b)
    for k, i in enumerate(ids_r):
        ctx_r.set_w(i, ws[k])
    for k, i in enumerate(ids_r):
        s1, C1, st1, _ = ctx_r.rve_solve([i], torch.tensor(b.Fbar[k:k + 1], device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(s1.cpu().numpy()[0], outs_a[0][0][k])
        assert np.array_equal(C1.cpu().numpy()[0], outs_a[0][1][k])
    ctx_r.close()


def test_admit_evict_and_refusals(torch):
    """fe2_rve_admit / fe2_rve_evict directly: a defined RVE is unusable until
    admitted, keeps its w~ across eviction, and the budget refuses what cannot
    fit."""
    from paper_2312_12771_gb300.fe2 import Fe2Context, Fe2Error, FE2_ERR_BUDGET, FE2_ERR_ARG
    b, ws = _case()
    ctx = Fe2Context(dim=2, precision="mixed")
    ids = ctx.define_batch(b.subset([1]))              # one RVE of 24^2
    ctx.set_w(ids[0], ws[1])
    F = torch.tensor(b.Fbar[1:2], device="cuda")
    with pytest.raises(Fe2Error) as ei:
        ctx.rve_solve(ids, F)
    assert ei.value.status == FE2_ERR_ARG
    ctx.admit(ids)
    s1 = [t.clone() for t in ctx.rve_solve(ids, F)]
    w1 = ctx.export(ids[0], 3, 24)
    assert np.array_equal(w1, ws[1])
    ctx.evict(ids)
    assert ctx.resident(ids[0]) == 0
    ctx.admit(ids)
    s2 = ctx.rve_solve(ids, F)
    torch.cuda.synchronize()
    assert torch.equal(s1[0], s2[0]) and torch.equal(s1[1], s2[1])
    ctx.close()
    ctx = Fe2Context(dim=2, precision="mixed", hbm_budget_bytes=100_000)   # less than one slot
    ids = ctx.define_batch(b.subset([1]))
    with pytest.raises(Fe2Error) as ei:
        ctx.admit(ids)
    assert ei.value.status == FE2_ERR_BUDGET
    ctx.close()
