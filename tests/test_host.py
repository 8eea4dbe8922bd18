"""Host-side logic of the product package, checked on the CPU against the
oracle's own, independently written, mesh generators and against invariants
of the bench's bookkeeping."""
import numpy as np
import pytest

from oracle import fe2_oracle as O
from paper_2312_12771_gb300 import workloads as W


@pytest.mark.parametrize("shape", [(1, 1), (3, 2), (5, 4)])
def test_q4_macro_mesh_matches_the_oracle(shape):
    from paper_2312_12771_gb300.driver import macro_mesh
    X, conn, fixed = macro_mesh(*shape)
    Xo, co, bo = O.macro_mesh(*shape)
    assert np.array_equal(X, Xo) and np.array_equal(conn, co)
    assert np.array_equal(np.nonzero(fixed[::2])[0], bo)
    assert np.array_equal(fixed[::2], fixed[1::2])


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 4), (4, 4, 4)])
def test_hex8_macro_mesh_matches_the_oracle(shape):
    from paper_2312_12771_gb300.driver import macro_mesh3
    X, conn, fixed = macro_mesh3(*shape)
    Xo, co, bo = O.macro_mesh3(*shape)
    assert np.array_equal(X, Xo) and np.array_equal(conn, co)
    assert np.array_equal(np.nonzero(fixed[::3])[0], bo)
    # positive Jacobian at every macro Gauss point, volume of the box
    _, etas, _ = O.macro_gauss(X, conn)
    assert (etas > 0).all() and abs(etas.sum() - 1.0) < 1e-12


def test_serving_sizes_and_arrivals_are_seeded_and_well_formed():
    s1, s2 = W.serving_sizes(3, 500), W.serving_sizes(3, 500)
    assert np.array_equal(s1, s2) and set(np.unique(s1)) <= {16, 24, 32, 48}
    a = W.poisson_arrivals(3, 2000, rate=1000.0)
    assert (np.diff(a) > 0).all()
    # mean inter-arrival time of a Poisson process of rate 1000 / s
    assert abs(np.diff(a).mean() - 1e-3) < 1e-4


def test_reference_arm_prints_the_contract_line():
    """``bench.py --impl reference`` (the FP64 oracle on the host cores) prints one
    JSON line with the keys of the bench contract, on a small workload."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--rves", "64", "--N", "8", "--cpu-sample", "8"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["config"]["N"] == 8 and d["config"]["rves_per_gpu"] == 64


def test_clock_sampler_summary_reports_median_and_throttle_reasons():
    """The bench's clock record: median SM clock under load, max clock, and the
    throttle reasons seen as Active in any sample (parsed from nvidia-smi CSV)."""
    import bench
    cs = bench.ClockSampler()
    rows = ["0, 2070, 2070, 150.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 180.4, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 170.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    cs.f.write("\n".join(rows) + "\n")
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"] and abs(s["power_w_max"] - 180.4) < 1e-9
    empty = bench.ClockSampler()
    assert empty.summary()["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("d,N", [(2, 6), (2, 8), (2, 9), (3, 3), (3, 4)])
def test_symbolic_column_counts_match_the_oracle_factor(d, N):
    """The work count of the band factor: the symbolic factorisation of K_mm in the
    folded periodic ordering against the nonzero pattern of the Cholesky factor of
    the oracle's K_mm (natural order, permuted).  Every numeric nonzero lies in the
    symbolic pattern, the half bandwidth is 4N + 5 in 2D, and the counts agree up
    to the rare entries that cancel exactly."""
    from paper_2312_12771_gb300 import workcount as WC
    rng = np.random.default_rng(N)
    ph = (rng.random(N ** d) < 0.4).astype(np.uint8)
    mat = W.linear_mat(1.0, 0.3, 10.0, 0.3)
    K = O.rve_solve(N, d, ph, mat, np.eye(d))["K_mm"]
    nm = K.shape[0]
    perm = np.zeros(nm, int)
    for p in range(1, N ** d):
        g = [(p // N ** k) % N for k in range(d)]
        q = sum(WC.fold_pos(g[k], N) * N ** k for k in range(d))
        for c in range(d):
            perm[d * (p - 1) + c] = d * (q - 1) + c
    Kf = np.zeros_like(K)
    Kf[np.ix_(perm, perm)] = K
    L = np.linalg.cholesky(Kf)
    sym = WC.column_structures(N, d)
    num_total = 0
    for j in range(nm):
        rows = np.nonzero(L[j + 1:, j])[0] + j + 1
        assert set(rows.tolist()) <= set(sym[j].tolist()), j
        num_total += len(rows)
    sym_total = int(WC.column_counts(N, d).sum())
    assert num_total <= sym_total <= 1.01 * num_total
    kd = max(int(c[-1]) - j for j, c in enumerate(sym) if len(c))
    if d == 2:
        assert kd == 4 * N + 5


def test_serving_tuner_choice_rule():
    """The serving tuner's pick from a measured table: the best capacity with no
    slack; within a slack, the smallest batch limit, then the fewest lanes."""
    from paper_2312_12771_gb300.tune import choose_server
    table = [{"max_batch": mb, "lanes": ln, "mixed": False, "capacity": c}
             for mb, ln, c in ((128, 2, 62.0), (128, 4, 78.8), (256, 3, 81.1), (256, 4, 82.5),
                               (512, 2, 74.1), (512, 4, 80.8))]
    best, top = choose_server(table)
    assert top == 82.5 and (best["max_batch"], best["lanes"]) == (256, 4)
    best, _ = choose_server(table, slack=0.05)
    assert (best["max_batch"], best["lanes"]) == (128, 4)
    best, _ = choose_server(table, slack=0.02)
    assert (best["max_batch"], best["lanes"]) == (256, 3)
    best, _ = choose_server(table, slack=1.0)
    assert (best["max_batch"], best["lanes"]) == (128, 2)
