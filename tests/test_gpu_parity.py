"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative error per RVE <= 1e-10 on the FP64 path and <= 1e-8 on
the mixed path (FP32 factor + FP64 refinement), for sigma_eff and Cbar;
reduced operators (K_mm, r_m, K_mM, K_MM, Pint) are FP64 on both paths and
must agree to 1e-13.  Relative error of sigma uses the floor
||Cbar_ref|| * ||Fbar - I|| so that a near-zero stress is not divided by ~0.
"""
import numpy as np
import pytest

from oracle import fe2_oracle as O
from paper_2312_12771_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-8}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12771_gb300 import build
    build.build()
    return t


def ctx_for(torch, precision, **kw):
    from paper_2312_12771_gb300.fe2 import Fe2Context
    return Fe2Context(dim=2, precision=precision, **kw)


def oracle_batch(batch, idx, w=None):
    out = []
    for k in idx:
        out.append(O.rve_solve(int(batch.N[k]), batch.d, batch.phase[k], batch.mat[k], batch.Fbar[k],
                               None if w is None else w[k]))
    return out


def sig_floor(ref):
    return np.linalg.norm(ref["Cbar"]) * np.linalg.norm(ref["Fbar_in"] - np.eye(2))


def check(batch, sig, Cb, st, refs, idx, tol):
    sig = sig.cpu().numpy()
    Cb = Cb.cpu().numpy()
    st = st.cpu().numpy()
    worst = 0.0
    for j, k in enumerate(idx):
        assert st[k] == 0, f"rve {k} status {st[k]}"
        ref = refs[j]
        eC = O.rel_err(Cb[k], ref["Cbar"])
        floor = np.linalg.norm(ref["Cbar"]) * np.linalg.norm(batch.Fbar[k] - np.eye(2))
        eS = O.rel_err(sig[k], ref["sigma_eff"], floor)
        worst = max(worst, eC, eS)
        assert eC <= tol, f"rve {k}: Cbar rel err {eC:.3e}"
        assert eS <= tol, f"rve {k}: sigma rel err {eS:.3e}"
    return worst


# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_laminate_closed_form_on_gpu(torch, precision):
    b = W.laminate_batch(64, 8)
    ctx = ctx_for(torch, precision)
    ids = ctx.register_batch(b)
    F = torch.tensor(b.Fbar, device="cuda")
    sig, Cb, st, err = ctx.rve_solve(ids, F)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    C = Cb.cpu().numpy()
    # Voigt [xx,yy,xy]: C11 = C[0,0], C22 = C[3,3], C12 = C[0,3], C66 = C[1,1]
    tol = TOL[precision] * 10
    assert np.allclose(C[:, 0, 0], 6.49350649350649, rtol=tol, atol=0)
    assert np.allclose(C[:, 3, 3], 2.44755244755245, rtol=tol, atol=0)
    assert np.allclose(C[:, 0, 3], 1.04895104895105, rtol=tol, atol=0)
    assert np.allclose(C[:, 1, 1], 0.699300699300699, rtol=tol, atol=0)
    s = sig.cpu().numpy()
    assert np.allclose(s[:, 0], 6.49350649350649e-3, rtol=tol, atol=0)
    assert np.allclose(s[:, 3], 1.04895104895105e-3, rtol=tol, atol=0)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [3, 5, 12])
def test_fiber_linear_parity(torch, precision, N):
    b = W.fiber_batch(6, N, dF_scale=2e-3)
    ctx = ctx_for(torch, precision)
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    idx = list(range(b.nrve))
    check(b, sig, Cb, st, oracle_batch(b, idx), idx, TOL[precision])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_neohooke_parity_with_fluctuation(torch, precision):
    """NH inclusions at a finite stretch, with a nonzero fluctuation state."""
    N = 10
    b = W.inclusion_batch(5, N, stretch=1.08)
    b.Fbar = W.perturbed_F(b, 7, 0.02)
    rng = np.random.default_rng(1)
    ws = [1e-3 * rng.standard_normal(2 * (N * N - 1)) for _ in range(b.nrve)]
    ctx = ctx_for(torch, precision)
    ids = ctx.register_batch(b)
    for k, i in enumerate(ids):
        ctx.set_w(i, ws[k])
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    idx = list(range(b.nrve))
    check(b, sig, Cb, st, oracle_batch(b, idx, ws), idx, TOL[precision])


@pytest.mark.parametrize("model", ["linear", "nh"])
def test_reduced_operator_entrywise(torch, model):
    """K_mm, r_m, K_mM, K_MM, Pint after the fused kernel and after the split
    assemble/reduce calls equal the oracle's T^T K T etc. entry by entry."""
    N = 7
    if model == "linear":
        b = W.fiber_batch(3, N, dF_scale=1e-2)
    else:
        b = W.inclusion_batch(3, N, stretch=1.1)
        b.Fbar = W.perturbed_F(b, 3, 0.03)
    rng = np.random.default_rng(5)
    ws = [2e-3 * rng.standard_normal(2 * (N * N - 1)) for _ in range(b.nrve)]
    ctx = ctx_for(torch, "fp64")
    ids = ctx.register_batch(b)
    for k, i in enumerate(ids):
        ctx.set_w(i, ws[k])
    F = torch.tensor(b.Fbar, device="cuda")
    refs = oracle_batch(b, range(b.nrve), ws)
    for path in ["fused", "split"]:
        if path == "fused":
            ctx.rve_solve(ids, F)
        else:
            ctx.micro_assemble(ids, F)
            ctx.nullspace_reduce(ids)
        torch.cuda.synchronize()
        for k, i in enumerate(ids):
            ref = refs[k]
            K = ctx.export(i, 0, N)
            scale = np.abs(ref["K_mm"]).max()
            assert np.abs(K - ref["K_mm"]).max() <= 1e-13 * scale, path
            assert np.abs(K - K.T).max() <= 1e-13 * scale
            r = ctx.export(i, 1, N)
            assert np.abs(r - ref["r_m"]).max() <= 1e-13 * max(1.0, np.abs(ref["r_m"]).max()) * scale, path
            KmM = ctx.export(i, 2, N)
            assert np.abs(KmM - ref["K_mM"]).max() <= 1e-13 * np.abs(ref["K_mM"]).max(), path
            mm = ctx.export(i, 4, N)
            assert np.abs(mm[:16] - ref["K_MM"].ravel()).max() <= 1e-13 * np.abs(ref["K_MM"]).max(), path
            assert np.abs(mm[16:] - ref["Pint"]).max() <= 1e-13 * max(1.0, np.abs(ref["Pint"]).max()), path


def test_split_and_fused_paths_agree_bitwise(torch):
    b = W.inclusion_batch(4, 9, stretch=1.05)
    ctx = ctx_for(torch, "mixed")
    ids = ctx.register_batch(b)
    F = torch.tensor(b.Fbar, device="cuda")
    s1, C1, st1, _ = ctx.rve_solve(ids, F)
    s1, C1 = s1.clone(), C1.clone()
    ctx.micro_assemble(ids, F)
    ctx.nullspace_reduce(ids)
    s2, C2, st2, _ = ctx.condense(ids)
    torch.cuda.synchronize()
    assert torch.equal(s1, s2) and torch.equal(C1, C2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fiber32_full_batch_sampled(torch, precision):
    """The bench workload: 4096 RVEs, 32x32 fiber, checked on sampled RVEs."""
    b = W.fiber_batch(4096, 32, dF_scale=1e-3)
    ctx = ctx_for(torch, precision)
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    idx = [0, 1, 777, 2048, 4001, 4095]
    w = check(b, sig, Cb, st, oracle_batch(b, idx), idx, TOL[precision])
    print(f"{precision}: worst sampled rel err {w:.3e}")
    # properties that hold for every RVE: major symmetry and the Voigt bound
    C = Cb.cpu().numpy()
    asym = np.abs(C - C.transpose(0, 2, 1)).max() / np.abs(C).max()
    assert asym <= TOL[precision]


def test_uneven_sizes_in_one_batch_match_alone(torch):
    """RVEs of different N in one call give the same result as alone."""
    parts = [W.inclusion_batch(2, N, stretch=1.05) for N in (6, 9, 13, 16)]
    N = np.concatenate([p.N for p in parts])
    phases = sum([p.phase for p in parts], [])
    mat = np.concatenate([p.mat for p in parts])
    F = np.concatenate([p.Fbar for p in parts])
    mixed = W.RveBatch(2, N, phases, mat, F)
    ctx = ctx_for(torch, "mixed")
    ids = ctx.register_batch(mixed)
    s_all, C_all, st, _ = ctx.rve_solve(ids, torch.tensor(F, device="cuda"))
    s_all, C_all = s_all.clone(), C_all.clone()
    for k, i in enumerate(ids):
        s1, C1, _, _ = ctx.rve_solve([i], torch.tensor(F[k:k + 1], device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(s1[0], s_all[k]) and torch.equal(C1[0], C_all[k])
    idx = list(range(mixed.nrve))
    check(mixed, s_all, C_all, st, oracle_batch(mixed, idx), idx, TOL["mixed"])


def test_macro_step_update_matches_oracle(torch):
    """w~ <- w~ - (x_r + X_M : dFbar) with the resident X_M, x_r."""
    N = 8
    b = W.inclusion_batch(3, N, stretch=1.1)
    ctx = ctx_for(torch, "fp64")
    ids = ctx.register_batch(b)
    ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    dF = np.array([[[1e-2, 2e-3], [-1e-3, -5e-3]]] * b.nrve)
    ctx.macro_step(ids, torch.tensor(dF, device="cuda"))
    torch.cuda.synchronize()
    for k, i in enumerate(ids):
        ref = O.rve_solve(N, 2, b.phase[k], b.mat[k], b.Fbar[k])
        w_ref = -(ref["x_r"] + ref["X_M"] @ dF[k].ravel())
        w = ctx.export(i, 3, N)
        assert np.abs(w - w_ref).max() <= 1e-10 * np.abs(w_ref).max()


def test_deterministic_repeat(torch):
    b = W.fiber_batch(64, 16)
    ctx = ctx_for(torch, "mixed")
    ids = ctx.register_batch(b)
    F = torch.tensor(b.Fbar, device="cuda")
    a = [t.clone() for t in ctx.rve_solve(ids, F)]
    c = ctx.rve_solve(ids, F)
    torch.cuda.synchronize()
    for x, y in zip(a, c):
        assert torch.equal(x, y)


def test_status_nan_and_not_pd(torch):
    b = W.fiber_batch(3, 6)
    b.mat[1, 0, 1] = -1.0     # negative Young's modulus in the matrix: indefinite K_mm
    ctx = ctx_for(torch, "fp64")
    ids = ctx.register_batch(b)
    F = b.Fbar.copy()
    F[2, 0, 0] = np.nan
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(F, device="cuda"))
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[0] == 0 and st[1] == 4 and st[2] == 5


def test_argument_errors(torch):
    from paper_2312_12771_gb300.fe2 import Fe2Error
    b = W.fiber_batch(2, 6)
    ctx = ctx_for(torch, "mixed")
    ids = ctx.register_batch(b)
    F = torch.tensor(b.Fbar, device="cuda")
    with pytest.raises(Fe2Error):
        ctx.rve_solve([ids[0], ids[0]], F)           # duplicate id
    with pytest.raises(Fe2Error):
        ctx.rve_solve([12345], F[:1])                # unknown id
    with pytest.raises(Fe2Error):
        ctx.nullspace_reduce(ids)                    # no element data yet


def test_budget_admission(torch):
    """Registration is refused (nothing admitted) once the HBM budget would be
    exceeded, and admitted again after a release frees room."""
    from paper_2312_12771_gb300.fe2 import Fe2Error, FE2_ERR_BUDGET
    ctx = ctx_for(torch, "mixed", hbm_budget_bytes=0)
    per = ctx.rve_bytes(16)          # persistent state + one workspace slot
    ctx.close()
    ctx = ctx_for(torch, "mixed", hbm_budget_bytes=int(per * 3))
    ids = ctx.register_batch(W.fiber_batch(3, 16))
    with pytest.raises(Fe2Error) as ei:
        ctx.register_batch(W.fiber_batch(10, 16))
    assert ei.value.status == FE2_ERR_BUDGET
    # the refused call admitted nothing: the three RVEs still solve
    b = W.fiber_batch(3, 16)
    sig, Cb, st, _ = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    ctx.release(ids)
    ctx.register_batch(W.fiber_batch(2, 16))      # fits again after release


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_monolithic_newton_matches_oracle(torch, precision):
    """Load-stepped monolithic Newton (macro 2x2 Q4, 16 NH RVEs with random
    inclusions, uniaxial stretch 1.1 in 2 steps): converged per-Gauss-point
    Pbar and Cbar, nodal positions and Newton iteration counts match the
    oracle's monolithic scheme."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    N = 6
    X, conn, fixed = macro_mesh(2, 2)
    b = W.inclusion_batch(16, N, stretch=1.0)
    ctx = ctx_for(torch, precision, refine_tol=1e-14, max_refine=2)
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    Ff = np.diag([1.1, 1.0])
    log = fe.run(Ff, 2, tol_macro=1e-10, tol_micro=1e-10)
    st = fe.state()
    rves = [dict(N=N, phase=b.phase[k], mat=b.mat[k]) for k in range(16)]
    out, iters, q = O.monolithic_fe2(O.macro_mesh(2, 2), rves, Ff, n_steps=2, tol_macro=1e-10, tol_micro=1e-10)
    assert log.iters == iters
    tol = TOL[precision]
    for k in range(16):
        assert O.rel_err(st["Pbar"][k], out[k]["Pbar"]) <= tol
        assert O.rel_err(st["Cbar"][k], out[k]["Cbar"]) <= tol
    assert np.abs(fe.ctx.macro_get_positions() - q).max() <= 1e-12


def test_macro_patch_test_on_gpu(torch):
    """Homogeneous RVEs and affine Dirichlet data: every Gauss point converges
    to Fbar = F_final and the nodal positions are affine."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    X, conn, fixed = macro_mesh(3, 2)
    m = np.array([[1, 1.0, 10.0, 0], [1, 1.0, 10.0, 0]])
    b = W.RveBatch(2, np.full(24, 4, np.int32), [np.zeros(16, np.uint8)] * 24, np.repeat(m[None], 24, 0),
                   np.repeat(np.eye(2)[None], 24, 0))
    ctx = ctx_for(torch, "mixed")
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    Ff = np.array([[1.08, 0.03], [0.0, 0.96]])
    fe.run(Ff, 2, tol_macro=1e-11, tol_micro=1e-11)
    st = fe.state()
    assert np.abs(st["Fbar"] - Ff[None]).max() < 1e-12
    assert np.abs(fe.ctx.macro_get_positions() - X @ Ff.T).max() < 1e-12


def test_serving_results_equal_alone_and_in_the_mix(torch):
    """Continuous batching: requests of uneven sizes (16, 24, 32 and 48 squared)
    served in overlapping batches give bit-identical sigma/Cbar to solving each
    RVE alone, and every request completes with a latency."""
    from paper_2312_12771_gb300.serve import Server, simulate
    sizes = W.serving_sizes(11, 48)
    b = W.inclusion_batch(48, sizes, stretch=1.02)
    ctx = ctx_for(torch, "mixed")
    ids = ctx.register_batch(b)
    srv = Server(ctx, max_batch=8, lanes=2)
    arrivals = W.poisson_arrivals(3, 48, rate=2000.0)
    res, p50, p99, thr = simulate(srv, np.asarray(ids), b.Fbar, arrivals)
    assert len(res["tickets"]) == 48 and (res["status"] == 0).all()
    assert p99 >= p50 > 0
    order = np.argsort(res["tickets"])
    for j, k in enumerate(order):
        s1, C1, st1, _ = ctx.rve_solve([ids[j]], torch.tensor(b.Fbar[j:j + 1], device="cuda"))
        torch.cuda.synchronize()
        assert np.array_equal(res["sigma"][k], s1.cpu().numpy()[0])
        assert np.array_equal(res["Cbar"][k], C1.cpu().numpy()[0])
    srv.close()


def test_serving_graph_replay_equals_direct_launches(torch):
    """A lane replays its captured CUDA graph for a batch shape it has seen
    before; the replayed batches give bit-identical sigma/Cbar to the same
    requests launched kernel by kernel."""
    from paper_2312_12771_gb300.serve import Server
    sizes = W.serving_sizes(5, 32)
    b = W.inclusion_batch(32, sizes, stretch=1.03)
    ctx = ctx_for(torch, "mixed")
    ids = np.asarray(ctx.register_batch(b))
    out = {}
    for graphs in (True, False):
        srv = Server(ctx, max_batch=8, lanes=2, graphs=graphs)
        got = []
        for _ in range(3):                     # the same burst three times
            tk = srv.submit(ids, b.Fbar)
            t, sig, Cb, st, _ = srv.drain()
            assert (st == 0).all() and len(t) == len(ids)
            pos = {int(x): j for j, x in enumerate(tk)}
            order = np.argsort([pos[int(x)] for x in t])
            got.append((sig[order], Cb[order]))
        cap, rep = srv.graph_stats()
        if graphs:
            assert cap > 0 and rep > 0, (cap, rep)
        else:
            assert cap == 0 and rep == 0
        srv.close()
        for s, c in got[1:]:
            assert np.array_equal(s, got[0][0]) and np.array_equal(c, got[0][1])
        out[graphs] = got[0]
    assert np.array_equal(out[True][0], out[False][0])
    assert np.array_equal(out[True][1], out[False][1])


def ctx3(torch, precision, **kw):
    from paper_2312_12771_gb300.fe2 import Fe2Context
    return Fe2Context(dim=3, precision=precision, **kw)


def check3(batch, sig, Cb, st, idx, tol, w=None):
    sig, Cb, st = sig.cpu().numpy(), Cb.cpu().numpy(), st.cpu().numpy()
    worst = 0.0
    for k in idx:
        assert st[k] == 0, f"rve {k} status {st[k]}"
        ref = O.rve_solve(int(batch.N[k]), 3, batch.phase[k], batch.mat[k], batch.Fbar[k])
        eC = O.rel_err(Cb[k], ref["Cbar"])
        floor = np.linalg.norm(ref["Cbar"]) * np.linalg.norm(batch.Fbar[k] - np.eye(3))
        eS = O.rel_err(sig[k], ref["sigma_eff"], floor)
        worst = max(worst, eC, eS)
        assert eC <= tol and eS <= tol, (k, eC, eS)
    return worst


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [3, 4])
def test_hex8_parity_small(torch, precision, N):
    """Hex8 RVEs (3D, periodic, corner pinned): NH sphere inclusion under shear
    and linear random phases, against the oracle."""
    b = W.sphere_batch(3, N, gamma=0.05)
    rng = np.random.default_rng(N)
    lin = W.RveBatch(3, np.full(3, N, np.int32), [(rng.random(N ** 3) < 0.4).astype(np.uint8) for _ in range(3)],
                     np.repeat(W.linear_mat(1.0, 0.3, 8.0, 0.25)[None], 3, 0),
                     np.repeat((np.eye(3) + 1e-3 * rng.standard_normal((3, 3)))[None], 3, 0))
    for batch in (b, lin):
        ctx = ctx3(torch, precision)
        ids = ctx.register_batch(batch)
        sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(batch.Fbar, device="cuda"))
        torch.cuda.synchronize()
        check3(batch, sig, Cb, st, range(batch.nrve), TOL[precision])
        ctx.close()


def test_hex8_homogeneous_recovers_local_law(torch):
    N = 4
    m = np.array([[1, 1.3, 11.0, 0], [1, 1.3, 11.0, 0]])
    F = np.eye(3) + np.array([[0.05, 0.02, -0.01], [0.0, -0.03, 0.04], [0.01, 0.0, 0.02]])
    b = W.RveBatch(3, np.array([N], np.int32), [np.zeros(N ** 3, np.uint8)], m[None], F[None])
    ctx = ctx3(torch, "mixed")
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    P, A = O.material(F[None], m[0], 3)
    assert np.abs(Cb.cpu().numpy()[0] - A[0].reshape(9, 9)).max() <= 1e-10 * np.abs(A).max()
    assert np.abs(sig.cpu().numpy()[0] - P[0].ravel()).max() <= 1e-10 * np.abs(P).max()


def test_hex8_config5_rve_sampled(torch):
    """The 3D workload RVE: 8^3 Hex8, centred sphere (vf 0.2), mu_i/mu_m = 10,
    simple shear gamma = 0.02; mixed path against the oracle on sampled RVEs."""
    b = W.sphere_batch(32, 8, gamma=0.02)
    b.Fbar = W.perturbed_F(b, 9, 2e-3)
    ctx = ctx3(torch, "mixed")
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    w = check3(b, sig, Cb, st, [0, 17, 31], TOL["mixed"])
    print(f"hex8 8^3 worst sampled rel err {w:.3e}")


def test_hex8_uneven_sizes_in_one_batch(torch):
    """One launch over Hex8 RVEs of 8^3 (kd = 440, wide-band factor, lane-split
    backward dot products) and of 3^3 and 4^3 (kd = 80, 128): every RVE matches
    the oracle, so the narrow bands are also correct on the wide code path.
    Mixed path only: registration refuses kd = 440 on the FP64 path, whose
    factor would not fit in shared memory."""
    precision = "mixed"
    a = W.sphere_batch(1, 8, gamma=0.03)
    rng = np.random.default_rng(4)
    Ns = [8, 3, 4, 3]
    phases = [a.phase[0]] + [(rng.random(n ** 3) < 0.4).astype(np.uint8) for n in Ns[1:]]
    b = W.RveBatch(3, np.array(Ns, np.int32), phases, np.repeat(a.mat[:1], 4, 0),
                   np.repeat(a.Fbar[:1], 4, 0))
    b.Fbar = W.perturbed_F(b, 6, 2e-3)
    ctx = ctx3(torch, precision)
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    check3(b, sig, Cb, st, range(4), TOL[precision])
    ctx.close()


def test_hex8_macro_patch_test_on_gpu(torch):
    """Hex8 macro mesh 6^3 (375 free DOFs, 12 panels of the blocked macro factor)
    with identical homogeneous RVEs and affine Dirichlet data: every Gauss point
    converges to Fbar = F_final and the nodal positions are affine."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh3
    X, conn, fixed = macro_mesh3(6, 6, 6)
    n = 8 * len(conn)
    m = np.array([[1, 1.0, 10.0, 0], [1, 1.0, 10.0, 0]])
    b = W.RveBatch(3, np.full(n, 3, np.int32), [np.zeros(27, np.uint8)] * n, np.repeat(m[None], n, 0),
                   np.repeat(np.eye(3)[None], n, 0))
    ctx = ctx3(torch, "mixed")
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    Ff = np.array([[1.05, 0.02, 0.0], [0.0, 0.97, 0.01], [0.03, 0.0, 1.02]])
    fe.run(Ff, 2, tol_macro=1e-11, tol_micro=1e-11)
    st = fe.state()
    assert np.abs(st["Fbar"] - Ff[None]).max() < 1e-12
    assert np.abs(fe.ctx.macro_get_positions() - X @ Ff.T).max() < 1e-12
    ctx.close()


def _macro_problem(d, shape, seed):
    """Structured Q4 / Hex8 macro mesh with its interior nodes moved by up to
    0.2 h, boundary nodes fixed."""
    from paper_2312_12771_gb300.driver import macro_mesh, macro_mesh3
    X, conn, fixed = macro_mesh(*shape) if d == 2 else macro_mesh3(*shape)
    rng = np.random.default_rng(seed)
    inner = fixed.reshape(-1, d)[:, 0] == 0
    X = X.copy()
    X[inner] += rng.uniform(-0.2, 0.2, (int(inner.sum()), d)) / max(shape)
    return X, conn, fixed, rng


@pytest.mark.parametrize("d,shape", [(2, (5, 5)), (2, (40, 30)), (3, (3, 3, 3)), (3, (6, 6, 5)),
                                     (3, (12, 12, 12))])
def test_macro_solve_matches_oracle(torch, d, shape):
    """One macro update (S7) for given sigma_eff and Cbar (random; Cbar SPD per
    Gauss point): dq from the blocked band Cholesky, dFbar_b = B_b dq and
    ||R_free|| equal a dense FP64 solve of the oracle's assembled system.  The
    cases cover a band narrower than one 32-column panel, many panels with a
    ragged last one, and (12^3 Hex8, 3993 DOFs, kd = 401) a trailing update of
    91 tiles."""
    from paper_2312_12771_gb300.fe2 import Fe2Context
    X, conn, fixed, rng = _macro_problem(d, shape, 5 + d)
    ctx = Fe2Context(dim=d, precision="fp64")
    ctx.macro_setup(X, conn, fixed)
    na, dd = 2 ** d, d * d
    ngp = na * len(conn)
    sig = rng.standard_normal((ngp, d, d))
    M = rng.standard_normal((ngp, dd, dd))
    Cb = np.einsum("bij,bkj->bik", M, M) + dd * np.eye(dd)[None]
    dF = torch.zeros((ngp, d, d), dtype=torch.float64, device="cuda")
    rn = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.ones(1, dtype=torch.int32, device="cuda")
    ctx.macro_solve(torch.tensor(sig, device="cuda"), torch.tensor(Cb, device="cuda"), dF, rn, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    dq = ctx.macro_get_positions() - X
    grads, etas, _ = O.macro_gauss(X, conn)
    K, R = O.macro_system(conn, grads, etas, sig, Cb, d)
    free = fixed == 0
    ref = np.zeros(len(free))
    ref[free] = np.linalg.solve(K[np.ix_(free, free)], -R[free])
    ref = ref.reshape(-1, d)
    assert np.abs(dq - ref).max() <= 1e-10 * np.abs(ref).max()
    assert abs(float(rn.item()) - np.linalg.norm(R[free])) <= 1e-12 * np.linalg.norm(R[free])
    dFh = dF.cpu().numpy()
    dFr = np.stack([ref[conn[b // na]].T @ grads[b] for b in range(ngp)])
    assert np.abs(dFh - dFr).max() <= 1e-10 * np.abs(dFr).max()
    # a tangent that is not positive definite is reported, not factorised silently
    ctx.macro_solve(torch.tensor(sig, device="cuda"), torch.tensor(-Cb, device="cuda"), dF, rn, st)
    torch.cuda.synchronize()
    from paper_2312_12771_gb300.fe2 import FE2_ERR_NOT_PD
    assert int(st.item()) == FE2_ERR_NOT_PD
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hex8_monolithic_newton_matches_oracle(torch, precision):
    """3D monolithic Newton (macro 2x2x2 Hex8, 64 NH RVEs of 3^3 with random
    inclusions; the faces x = 0 and x = 1 carry the affine Dirichlet data
    F = I + 0.04 e1 (x) e1 + 0.03 e2 (x) e1 in 2 load steps, the other boundary
    nodes are free, so the macro field is not affine): converged Pbar, Cbar,
    positions and iteration counts match the oracle.  (A load that compresses
    the elements next to a face, started from w~ = 0 without a predictor,
    makes some heterogeneous 3^3 micro Hessians indefinite at the first
    iterate, on both sides.)"""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh3
    X, conn, fixed = macro_mesh3(2, 2, 2)
    onx = (np.abs(X[:, 0]) < 1e-12) | (np.abs(X[:, 0] - 1.0) < 1e-12)
    fixed = np.repeat(onx, 3).astype(np.uint8)
    N = 3
    b = W.inclusion_batch(64, N, d=3)
    ctx = ctx3(torch, precision, refine_tol=1e-14, max_refine=2)
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    Ff = np.eye(3)
    Ff[0, 0] += 0.04
    Ff[1, 0] = 0.03
    log = fe.run(Ff, 2, tol_macro=1e-10, tol_micro=1e-10)
    st = fe.state()
    rves = [dict(N=N, phase=b.phase[k], mat=b.mat[k]) for k in range(64)]
    out, iters, q = O.monolithic_fe2((X, conn, np.nonzero(onx)[0]), rves, Ff, n_steps=2,
                                     tol_macro=1e-10, tol_micro=1e-10)
    assert log.iters == iters
    tol = TOL[precision]
    for k in range(64):
        assert O.rel_err(st["Pbar"][k], out[k]["Pbar"]) <= tol
        assert O.rel_err(st["Cbar"][k], out[k]["Cbar"]) <= tol
    assert np.abs(fe.ctx.macro_get_positions() - q).max() <= 1e-11
    # the free faces moved: the solution is not the affine map of the Dirichlet data
    assert np.abs(q - X @ Ff.T).max() > 1e-4
    ctx.close()


def test_monolithic_newton_affine_predictor(torch):
    """With the affine predictor the converged state is the same fixed point
    (the predictor only changes the start value of each load step)."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    N = 6
    X, conn, fixed = macro_mesh(2, 2)
    b = W.inclusion_batch(16, N, stretch=1.0)
    Ff = np.diag([1.1, 1.0])
    states = []
    for pred in (False, True):
        ctx = ctx_for(torch, "fp64")
        fe = MonolithicFE2(ctx, X, conn, fixed, b)
        fe.run(Ff, 2, predictor=pred, tol_macro=1e-11, tol_micro=1e-11)
        states.append(fe.state())
        ctx.close()
    for k in range(16):
        assert O.rel_err(states[1]["Pbar"][k], states[0]["Pbar"][k]) <= 1e-9
        assert O.rel_err(states[1]["Cbar"][k], states[0]["Cbar"][k]) <= 1e-9


def test_bounded_wait_reports_timeout_and_context_survives(torch):
    """A device wait that can never complete gives up with FE2_ERR_TIMEOUT
    (no trap, no hang) and the context keeps working afterwards."""
    from paper_2312_12771_gb300.fe2 import FE2_ERR_TIMEOUT
    ctx = ctx_for(torch, "mixed")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ctx.lib.fe2_selftest_wait_timeout(ctx.h, C_ptr(st)) == 0
    torch.cuda.synchronize()
    assert int(st.item()) == FE2_ERR_TIMEOUT
    b = W.fiber_batch(2, 8)
    ids = ctx.register_batch(b)
    _, _, s2, _ = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    assert (s2.cpu().numpy() == 0).all()


def C_ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("N", [3, 8, 16, 20, 24, 30, 32])
def test_tensor_core_factor_parity(torch, N):
    """Mixed path with the tcgen05 (3xTF32) band factor against the oracle and
    against the CUDA-core FP32 factor.  N spans the kernels and operand shapes:
    one RVE per SM (N = 3, 8), two per SM with one 128-row tile (N = 16, 20,
    24), two row tiles without (N = 30) and with (N = 32) the corner tile
    beyond column 128."""
    b = W.fiber_batch(4, N, dF_scale=2e-3)
    out = {}
    for kern in ("tensor_core", "cuda_core"):
        ctx = ctx_for(torch, "mixed", factor=kern)
        ids = ctx.register_batch(b)
        ctx.profile(True)
        sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
        torch.cuda.synchronize()
        names = ctx.profile_read()
        assert ("band_factor_tc" in names) == (kern == "tensor_core"), names
        out[kern] = (sig.clone(), Cb.clone(), st.clone())
    idx = list(range(b.nrve))
    refs = oracle_batch(b, idx)
    for kern, (sig, Cb, st) in out.items():
        check(b, sig, Cb, st, refs, idx, TOL["mixed"])
    dC = (out["tensor_core"][1] - out["cuda_core"][1]).abs().max().item()
    assert dC <= 1e-8 * out["cuda_core"][1].abs().max().item()


def test_tensor_core_factor_mixed_sizes(torch):
    """The two-RVE-per-SM tensor-core factor with RVEs of 16^2, 24^2 and 32^2 in
    one launch (each CTA lays out its own band inside the launch's largest):
    every result against the oracle, and bitwise equal to the same RVE solved
    alone."""
    sizes = np.array([16, 24, 32, 24, 16, 32], np.int32)
    b = W.inclusion_batch(len(sizes), sizes, stretch=1.04)
    ctx = ctx_for(torch, "mixed", factor="tensor_core")
    ids = ctx.register_batch(b)
    F = torch.tensor(b.Fbar, device="cuda")
    sig, Cb, st, err = ctx.rve_solve(ids, F)
    torch.cuda.synchronize()
    idx = list(range(b.nrve))
    check(b, sig, Cb, st, oracle_batch(b, idx), idx, TOL["mixed"])
    for k in (0, 1, 2):
        s1, C1, _, _ = ctx.rve_solve(ids[k:k + 1], F[k:k + 1])
        torch.cuda.synchronize()
        assert torch.equal(C1[0], Cb[k]) and torch.equal(s1[0], sig[k])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_staggered_scheme_matches_oracle_and_monolithic(torch, precision):
    """Classical staggered FE^2 (Section 4.1) on the GPU: inner micro Newton to
    equilibrium in every macro iteration, macro step with the condensed tangent,
    micro states moved by Eq. (reduction).  Macro iteration counts and
    converged states match the oracle's staggered scheme, and the converged
    state is the monolithic scheme's (both solve the same discrete equations)."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    N = 6
    X, conn, fixed = macro_mesh(2, 2)
    b = W.inclusion_batch(16, N, stretch=1.0)
    Ff = np.diag([1.1, 1.0])
    ctx = ctx_for(torch, precision, refine_tol=1e-14, max_refine=2)
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    log = fe.run(Ff, 2, scheme="staggered", tol_macro=1e-10, tol_micro=1e-11)
    st = fe.state()
    q_s = fe.ctx.macro_get_positions()
    rves = [dict(N=N, phase=b.phase[k], mat=b.mat[k]) for k in range(16)]
    out, iters, micro, q = O.staggered_fe2(O.macro_mesh(2, 2), rves, Ff, n_steps=2, tol_macro=1e-10,
                                           tol_micro=1e-11)
    assert log.iters == iters
    assert log.micro_iters > 0
    tol = TOL[precision]
    for k in range(16):
        assert O.rel_err(st["Pbar"][k], out[k]["Pbar"]) <= tol
        assert O.rel_err(st["Cbar"][k], out[k]["Cbar"]) <= tol
    assert np.abs(q_s - q).max() <= 1e-11
    # same equilibrium as the monolithic scheme on the GPU
    ctx2 = ctx_for(torch, precision, refine_tol=1e-14, max_refine=2)
    fm = MonolithicFE2(ctx2, X, conn, fixed, b)
    fm.run(Ff, 2, tol_macro=1e-10, tol_micro=1e-10)
    sm = fm.state()
    assert np.abs(fm.ctx.macro_get_positions() - q_s).max() <= 1e-10
    for k in range(16):
        assert O.rel_err(sm["Cbar"][k], st["Cbar"][k]) <= 10 * tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("N", [6, 12])
def test_mooney_rivlin_cross_rve_parity(torch, precision, N):
    """Section 5.2 membrane RVE: the cross microstructure of the two
    Mooney-Rivlin materials at finite, non-symmetric Fbar."""
    b = W.cook_batch(5, N)
    rng = np.random.default_rng(7)
    b.Fbar = np.eye(2)[None] + 0.12 * rng.standard_normal((5, 2, 2))
    ctx = ctx_for(torch, precision)
    ids = ctx.register_batch(b)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(b.Fbar, device="cuda"))
    torch.cuda.synchronize()
    idx = list(range(b.nrve))
    check(b, sig, Cb, st, oracle_batch(b, idx), idx, TOL[precision])


def test_mooney_rivlin_is_2d_only(torch):
    from paper_2312_12771_gb300.fe2 import Fe2Context, Fe2Error
    ctx = Fe2Context(dim=3, precision="fp64")
    b = W.sphere_batch(1, 3)
    b.mat[:] = W.mooney_rivlin_mat(W.MEMBRANE_MATERIAL_1, W.MEMBRANE_MATERIAL_2)
    with pytest.raises(Fe2Error):
        ctx.register_batch(b)


@pytest.mark.parametrize("scheme", ["monolithic", "staggered"])
def test_cook_membrane_matches_oracle(torch, scheme):
    """Section 5.2 Cook's membrane on a 2x2 macro mesh with 6x6 cross RVEs:
    clamped left edge, traction (-5, 10) on the right edge in n_l = 2 load
    steps.  Newton iteration counts, tip position and converged Pbar, Cbar
    equal the oracle's (FP64 path)."""
    from paper_2312_12771_gb300.driver import MonolithicFE2
    X, conn, left, right = W.cook_mesh(2, 2)
    fixed = np.zeros(2 * len(X), np.uint8)
    for n in left:
        fixed[2 * n:2 * n + 2] = 1
    b = W.cook_batch(4 * len(conn), 6)
    ctx = ctx_for(torch, "fp64")
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    kw = dict(tol_macro=1e-9, tol_micro=1e-11) if scheme == "staggered" else dict(tol_macro=1e-9, tol_micro=1e-9)
    log = fe.run(np.eye(2), 2, scheme=scheme, traction=(right, W.MEMBRANE_TRACTION), **kw)
    st = fe.state()
    q = fe.ctx.macro_get_positions()
    rves = [dict(N=6, phase=b.phase[k], mat=b.mat[k]) for k in range(b.nrve)]
    fo = O.traction_load(X, right, W.MEMBRANE_TRACTION)
    if scheme == "monolithic":
        out, iters, q_ref = O.monolithic_fe2((X, conn, left), rves, np.eye(2), n_steps=2, fext=fo, **kw)
    else:
        out, iters, _, q_ref = O.staggered_fe2((X, conn, left), rves, np.eye(2), n_steps=2, fext=fo, **kw)
    assert log.iters == iters
    assert np.abs(q - q_ref).max() <= 1e-8 * np.abs(q_ref).max()
    for k in range(b.nrve):
        assert O.rel_err(st["Pbar"][k], out[k]["Pbar"]) <= 1e-9
        assert O.rel_err(st["Cbar"][k], out[k]["Cbar"]) <= 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_element_rve_piecewise_constant_basis_parity(torch, precision):
    """Eqs. (constSolution1), (constSolution2): element RVEs with four macro
    Gauss points (different Fbar, non-uniform weights) against the oracle's
    rve_solve_elem: the 16x16 coupled tangent and the four stresses."""
    from paper_2312_12771_gb300.fe2 import Fe2Context
    n, N = 6, 6
    b = W.inclusion_batch(n, N, stretch=1.0)
    rng = np.random.default_rng(13)
    F = np.eye(2)[None, None] + 0.06 * rng.standard_normal((n, 4, 2, 2))
    wq = rng.uniform(0.5, 1.5, (n, 4))
    wq /= wq.sum(axis=1, keepdims=True)
    ctx = Fe2Context(dim=2, precision=precision, basis="const")
    ids = ctx.register_batch(b)
    ctx.rve_set_quad_weights(ids, wq)
    sig, Cb, st, err = ctx.rve_solve(ids, torch.tensor(F, device="cuda"))
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    sig = sig.cpu().numpy().reshape(n, 4, 4)
    Cb = Cb.cpu().numpy()
    tol = TOL[precision]
    for k in range(n):
        ref = O.rve_solve_elem(N, 2, b.phase[k], b.mat[k], list(F[k]), wq[k])
        assert O.rel_err(Cb[k], ref["Cbar"]) <= tol
        floor = np.linalg.norm(ref["Cbar"]) * np.linalg.norm(F[k] - np.eye(2)[None])
        assert O.rel_err(sig[k], ref["sigma_eff"], floor) <= tol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_piecewise_constant_basis_newton_matches_oracle(torch, precision):
    """Monolithic Newton with one element RVE per macro element (macro 2x2
    Q4, NH inclusion RVEs 6x6, stretch 1.1 in 2 steps): iteration counts,
    nodal positions and converged Pbar, Cbar equal the oracle's."""
    from paper_2312_12771_gb300.driver import MonolithicFE2, macro_mesh
    from paper_2312_12771_gb300.fe2 import Fe2Context
    N = 6
    X, conn, fixed = macro_mesh(2, 2)
    b = W.inclusion_batch(len(conn), N, stretch=1.0)
    ctx = Fe2Context(dim=2, precision=precision, basis="const", refine_tol=1e-14, max_refine=2)
    fe = MonolithicFE2(ctx, X, conn, fixed, b)
    Ff = np.diag([1.1, 1.0])
    log = fe.run(Ff, 2, tol_macro=1e-10, tol_micro=1e-10)
    st = fe.state()
    rves = [dict(N=N, phase=b.phase[k], mat=b.mat[k]) for k in range(len(conn))]
    out, iters, q = O.monolithic_fe2_const(O.macro_mesh(2, 2), rves, Ff, n_steps=2, tol_macro=1e-10,
                                           tol_micro=1e-10)
    assert log.iters == iters
    tol = TOL[precision]
    for e in range(len(conn)):
        assert O.rel_err(st["Pbar"][4 * e:4 * e + 4], out[e]["Pbar"]) <= tol
        assert O.rel_err(st["Cbar"][e], out[e]["Cbar"]) <= tol
    assert np.abs(fe.ctx.macro_get_positions() - q).max() <= 1e-11
