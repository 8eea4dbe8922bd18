"""fe2_rve_solve_noalloc: the allocation-free entry point for callers that
cannot call cudaMalloc (a framework or plugin host that owns the device
allocator, or a real-time loop).  Its results must equal those of the
context-based fused entry point fe2_rve_solve (mixed path, no refinement)
within the mixed-path tolerance, on two calls in a row that reuse the same
device scratch array with different inputs.  This file is collected last so a
run that stops at the first failure has already run every other test; it
passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

from paper_2312_12771_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-8


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12771_gb300 import build
    build.build()
    from paper_2312_12771_gb300.fe2 import Fe2Context, rve_solve_noalloc

    batches = [W.inclusion_batch(12, 16, stretch=1.06), W.fiber_batch(9, 12, dF_scale=2e-3)]
    for b in batches:
        N = int(b.N[0])
        ctx = Fe2Context(dim=2, precision="mixed", max_refine=0)
        ids = ctx.register_batch(b)
        F = torch.tensor(b.Fbar, device="cuda")
        s_ref, C_ref, st_ref, _ = ctx.rve_solve(ids, F)
        phase = torch.tensor(np.stack(b.phase), dtype=torch.uint8, device="cuda")
        mat = torch.tensor(b.mat, device="cuda")
        out = (torch.full((b.nrve, 4), float("nan"), dtype=torch.float64, device="cuda"),
               torch.full((b.nrve, 4, 4), float("nan"), dtype=torch.float64, device="cuda"),
               torch.full((b.nrve,), -1, dtype=torch.int32, device="cuda"),
               torch.zeros(b.nrve, dtype=torch.float64, device="cuda"))
        sig, Cb, st, err = rve_solve_noalloc(N, phase, mat, F, out)
        torch.cuda.synchronize()
        # same status as the context path (OK, or NO_CONV where the estimate exceeds 1e-10)
        assert np.array_equal(st.cpu().numpy(), st_ref.cpu().numpy())
        assert set(np.unique(st.cpu().numpy())) <= {0, 6}
        sig, Cb = sig.cpu().numpy(), Cb.cpu().numpy()
        s_ref, C_ref = s_ref.cpu().numpy(), C_ref.cpu().numpy()
        for k in range(b.nrve):
            assert rel(Cb[k], C_ref[k]) <= TOL
            floor = np.linalg.norm(C_ref[k]) * np.linalg.norm(b.Fbar[k] - np.eye(2))
            assert np.linalg.norm(sig[k] - s_ref[k]) / max(np.linalg.norm(s_ref[k]), floor) <= TOL
        ctx.close()


def test_noalloc_rejects_bad_device_inputs_per_rve():
    """A phase index >= nphase and an unknown material model are found on the
    device: those RVEs get FE2_ERR_ARG, the others are solved as usual.  The
    mat tensor is a view into a larger buffer, so a missing check would read
    the padding row, not past an allocation."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12771_gb300 import build
    build.build()
    from paper_2312_12771_gb300.fe2 import Fe2Context, rve_solve_noalloc, FE2_ERR_ARG
    b = W.inclusion_batch(5, 12, stretch=1.04)
    N, n = 12, b.nrve
    ph = np.stack(b.phase).copy()
    ph[1, 7] = 2                            # nphase = 2: out of range
    mat_big = np.concatenate([b.mat, b.mat[:1]], axis=0)
    mat_big[3, 1, 0] = 7.0                  # unknown model code
    phase = torch.tensor(ph, dtype=torch.uint8, device="cuda")
    mat = torch.tensor(mat_big, device="cuda")[:n]
    F = torch.tensor(b.Fbar, device="cuda")
    out = (torch.zeros((n, 4), dtype=torch.float64, device="cuda"),
           torch.zeros((n, 4, 4), dtype=torch.float64, device="cuda"),
           torch.full((n,), -1, dtype=torch.int32, device="cuda"), None)
    sig, Cb, st, _ = rve_solve_noalloc(N, phase, mat, F, out)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[1] == FE2_ERR_ARG and st[3] == FE2_ERR_ARG
    good = [0, 2, 4]
    assert set(st[good]) <= {0, 6}
    ctx = Fe2Context(dim=2, precision="mixed", max_refine=0)
    ids = ctx.register_batch(b.subset(good))
    s_ref, C_ref, st_ref, _ = ctx.rve_solve(ids, F[good])
    torch.cuda.synchronize()
    C_ref = C_ref.cpu().numpy()
    for j, k in enumerate(good):
        assert rel(Cb.cpu().numpy()[k], C_ref[j]) <= TOL
    ctx.close()


def test_noalloc_capacity_and_argument_checks_on_gpu():
    """39 RVEs of 32 x 32 fit the scratch array (40 do not); the Python wrapper
    rejects tensors of the wrong dtype, shape or device before the call."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_12771_gb300 import build
    build.build()
    from paper_2312_12771_gb300.fe2 import Fe2Error, rve_solve_noalloc, FE2_ERR_BUDGET
    for n, ok in ((39, True), (40, False)):
        b = W.fiber_batch(n, 32, dF_scale=1e-3)
        phase = torch.tensor(np.stack(b.phase), dtype=torch.uint8, device="cuda")
        mat = torch.tensor(b.mat, device="cuda")
        F = torch.tensor(b.Fbar, device="cuda")
        out = (torch.zeros((n, 4), dtype=torch.float64, device="cuda"),
               torch.zeros((n, 4, 4), dtype=torch.float64, device="cuda"),
               torch.zeros((n,), dtype=torch.int32, device="cuda"),
               torch.zeros((n,), dtype=torch.float64, device="cuda"))
        if ok:
            rve_solve_noalloc(32, phase, mat, F, out)
            torch.cuda.synchronize()
            assert set(np.unique(out[2].cpu().numpy())) <= {0, 6}
        else:
            with pytest.raises(Fe2Error) as ei:
                rve_solve_noalloc(32, phase, mat, F, out)
            assert ei.value.status == FE2_ERR_BUDGET
    n = 2
    b = W.fiber_batch(n, 8)
    phase = torch.tensor(np.stack(b.phase), dtype=torch.uint8, device="cuda")
    mat = torch.tensor(b.mat, device="cuda")
    F = torch.tensor(b.Fbar, device="cuda")
    out = (torch.zeros((n, 4), dtype=torch.float64, device="cuda"),
           torch.zeros((n, 4, 4), dtype=torch.float64, device="cuda"),
           torch.zeros((n,), dtype=torch.int32, device="cuda"), None)
    with pytest.raises(ValueError):
        rve_solve_noalloc(8, phase, mat.float(), F, out)             # float32 materials
    with pytest.raises(ValueError):
        rve_solve_noalloc(8, phase.cpu(), mat, F, out)               # host tensor
    with pytest.raises(ValueError):
        rve_solve_noalloc(9, phase, mat, F, out)                     # phase is [n, 64], not [n, 81]
    with pytest.raises(ValueError):
        rve_solve_noalloc(8, phase, mat, F, (out[0], out[1], out[2].long(), None))   # int64 status
