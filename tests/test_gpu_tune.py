"""The autotuner (paper_2312_12771_gb300.tune): it picks a measured candidate,
its choice reproduces the candidate's results, and the cache answers a
repeated question without measuring again."""
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


def test_tune_factor_and_server_with_cache(torch, tmp_path):
    from paper_2312_12771_gb300 import tune
    from paper_2312_12771_gb300.fe2 import Fe2Context
    cache = str(tmp_path / "tune.json")
    b = W.inclusion_batch(16, 16, stretch=1.03)
    r1 = tune.tune_factor(b, cache=cache, reps=1)
    assert r1["best"] in r1["ms"] and not r1["cached"]
    assert tune.tune_factor(b, cache=cache)["cached"]
    sizes = np.array([16, 24] * 32, np.int32)
    s = W.inclusion_batch(64, sizes, stretch=1.03)
    ctx = Fe2Context(dim=2, precision="mixed")
    ids = np.asarray(ctx.register_batch(s))
    r2 = tune.tune_server(ctx, ids, s.Fbar, sizes, max_batches=(8, 32), lanes=(1, 2), mixed=(False, True),
                          cache=cache)
    assert len(r2["table"]) == 8 and r2["capacity"] == max(r["capacity"] for r in r2["table"])
    assert tune.tune_server(ctx, ids, s.Fbar, sizes, cache=cache)["cached"]
    # mixed-size batches give the same results as one size per batch
    from paper_2312_12771_gb300.serve import Server
    got = {}
    for mixed in (False, True):
        srv = Server(ctx, max_batch=16, lanes=2, mixed=mixed)
        tk = srv.submit(ids, s.Fbar)
        t, sig, Cb, st, _ = srv.drain()
        srv.close()
        pos = {int(x): j for j, x in enumerate(tk)}
        order = np.argsort([pos[int(x)] for x in t])
        got[mixed] = (sig[order], Cb[order])
        assert (st == 0).all()
    assert np.array_equal(got[False][0], got[True][0]) and np.array_equal(got[False][1], got[True][1])
    ctx.close()
